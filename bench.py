#!/usr/bin/env python
"""Throughput of the nonlinear Poisson-Boltzmann FEM-BEM Newton solve on GB300.

One step = one complete solve of the multi-charge sphere workload through the
C ABI: linear part (GMRES), Newton-Raphson with the cubic first iteration and
the automatic relaxation factor (batched residual evaluations), and the
solvation energy -- every row of the hot path.  The mesh is created and the
charges set before timing (inputs resident in HBM).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                  [--impl pbfb|reference]
  python bench.py --step farfield_f32|farfield_ff|farfield_f64|assemble|omega|gmres [--reps R]
                  [--workload small]   (one step of the solve, for profiler captures)

Beside the headline line's workload: the plain float64 GPU path timed over the same
number of solves ("fp64_gpu"), "full_formulation" (the paper's own formulation: FEM
over Omega_m and Omega_i, charges as point loads, lam_m from the Gamma_m equation, on
the same sphere meshed inside Gamma_m too), a serving run, and the CPU oracle.

--impl reference times the CPU oracle (the plain float64 restatement of the
method under oracle/) on bounded samples of the same workload, scaled to
solves/s with the oracle's own iteration counts.  Under torchrun (N > 1) every
rank runs independent replicas of the solve (no collective on the data path);
rank 0 prints.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "nonlinear PB solves/s and p99 ms, mixed vs FP64 GPU at ≤1e-5 rel energy err"
FP32_LANES = 128          # float32 FMA lanes per SM (Blackwell)
SM_MAX_MHZ = 2070.0       # GB300 maximum SM clock, used when nvidia-smi reports none
# algorithmic float32 work of one ordered far-field pair (FMA = 2): the fused single + double
# layer, about 20 flops for the Laplace kernel and 28 for the Yukawa kernel (its exponential
# factor and (1 + kappa r) term), with one rsqrt (and one exp) on the special-function unit
FLOP_PAIR = {"laplace": 20.0, "yukawa": 28.0}
# pbfb_newton_opts.residual_far: PBFB_FLOAT2 (float-float direct sum) or PBFB_MIXED (float32 operator)
RESIDUAL_FAR = {"float2": 2, "f32": 1}
GOLDEN = os.path.join(ROOT, "tests", "golden", "multi_charge_sphere.json")
# DRAM bytes (read + write) per launch on this workload, each from an ncu capture of the kernel
# (dram__bytes_read.sum + dram__bytes_write.sum): the packed float32 far field (source records
# read once) and the packed mutual float-float far field
NBODY_TRAFFIC = 2311424.0
FF2_TRAFFIC = 15.17e6
FF_TRAFFIC = 15.2e6
# float32 lane operations (FADD, FMUL, FFMA each 1; a packed instruction 2) per ordered pair that
# the float-float evaluation issues, counted by ncu on the packed mutual kernel: the emulation's
# cost, against 20 / 28 flops of the method's own arithmetic
FF_OPS_PAIR = {"laplace": 97.7, "yukawa": 145.7}
# the oracle's measured full solve of this workload on one host (x86-64, 8 cores: dense BEM
# set-up and the default-tolerance solve, written by tests/golden/make_golden.py), against which
# the sampled CPU model was checked once on that host
ORACLE_C2_MEASURED_HOST = "x86-64, 8 cores"
ORACLE_C2_MODEL_ON_THAT_HOST = 1047.0   # the model below with --cpu-sample 128 on that host: 16 % above


def workload_config(case, precision):
    if case.n_v != 72036:
        return {"workload": "single_charge_sphere (profiling case)", "n_vertices": int(case.n_v),
                "n_tets": int(case.n_t), "precision": precision}
    return {
        "workload": "multi_charge_sphere",
        "geometry": "solute sphere r=12 A, FEM shell to 24 A (17 geometric layers), "
                    "icosphere nu=20 on both surfaces",
        "n_vertices": int(case.n_v), "n_tets": int(case.n_t),
        "gamma_m_triangles": int(case.gm_tris.shape[0]), "gamma_s_triangles": int(case.gs_tris.shape[0]),
        "charges": "200 x (+-1 e) uniform in r<10 A, net -20 e (seed 2000)",
        "eps_in": case.eps_in, "eps_out": case.eps_out, "ionic_M": 0.1, "kappa_per_A": round(case.kappa, 6),
        "T_K": case.T, "precision": precision,
        "newton": "T3 first iteration, automatic omega (Newton on f_d), L_e 0.35, Tol_omega 0.1, "
                  "Tol_GR0 1e-3 -> Tol_GR 1e-6, Tol_NL 1e-3",
        "residual": "float-float far field at the first Newton step; later steps update it by linearity "
                    "(c += omega p, p = -Acal(0) Delta with the float32 operator) while the updates since the "
                    "last float-float evaluation sum to at most residual_update x ||Phi|| "
                    "(pbfb_newton_opts.residual_update; mixed_residual_every_step times it at 0)",
        "preconditioner": "flexible GMRES, block-triangular: dense float32 single-layer inverses on the "
                          "surface rows (built once per mesh and kappa), then 30 Jacobi-PCG iterations on "
                          "the FEM block",
        "l2": "flushed between timed steps (256 MiB write)",
    }


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, device, ws):
    """The largest of every rank's value (the job's time is its slowest replica's)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as tdist
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ws, steps, total_ms_max):
    """Solves per second of the whole job: every rank solved `steps` instances (replicas)."""
    return ws * steps / (total_ms_max / 1e3)


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.gpu = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def serving_cases(n, seed=5000):
    """Seeded serving requests, sphere or double helix by a fair coin, 2000-8000 triangles per
    surface (log-uniform), ionic strength U(0.01, 1) M, eps_in in {2, 4}.  Spheres: radius 12,
    shell to 24, 1-200 unit charges in r < 9.6; meshes of the same frequency are shared, so
    repeated geometries occur (as for repeated requests on one molecule).  Helices: 8-24 base
    pairs with their atoms' charges, shell to three Debye lengths beyond the surface."""
    import numpy as np
    from paper_2511_21713_gb300 import inputs
    rng = inputs.SplitMix64(seed)
    meshes, cases = {}, []
    for i in range(n):
        tri = 2000.0 * 4.0 ** rng.uniform()
        nu = max(10, min(20, int(round((tri / 20.0) ** 0.5))))
        ionic = 0.01 + 0.99 * rng.uniform()
        eps_in = (2.0, 4.0)[rng.below(2)]
        kappa = inputs.kappa_from_ionic_strength(ionic, 80.0, 300.0)
        if rng.below(2) == 0:
            nq = 1 + rng.below(200)
            q, z = inputs.ball_charges(nq, 9.6, rng.below(nq + 1), seed + 17 * i)
            if nu not in meshes:
                meshes[nu] = inputs.spherical_shell(nu, 12.0, 24.0, max(8, int(0.85 * nu)))
            xyz, tets, gm, gs = meshes[nu]
            cases.append(inputs.Case(f"serve{i}", xyz, tets, gm, gs, q, z, eps_in, 80.0, kappa, 300.0))
        else:
            nbp = 8 + rng.below(17)
            h = inputs.double_helix(n_bp=nbp, nu=nu, layers=max(8, int(0.6 * nu)), seed=seed + 31 * i,
                                    n_interior=62 * nbp, ionic=ionic, eps_in=eps_in)
            cases.append(h)
    return cases


def run_serving(pbfb, cases, max_inflight, budget, residual_update=0.0, precision=None, detail=False,
                residual_far="float2"):
    """Saturation run (all requests at t = 0) for capacity, then Poisson arrivals at 0.8x
    capacity; latency = arrival -> result (the request's own set-up included)."""
    import numpy as np
    from paper_2511_21713_gb300 import inputs

    def drain(sv, n, until=None):
        got = []
        while len(got) < n:
            got += sv.poll(64, 100000)
        return got

    precision = pbfb.MIXED if precision is None else precision
    opts = pbfb.default_opts(precision=precision, residual_update=residual_update,
                             residual_far=RESIDUAL_FAR[residual_far])
    sv = pbfb.Server(budget, max_inflight, cached_meshes=16)
    t0 = time.perf_counter()
    for i, c in enumerate(cases):
        sv.submit(c, i, opts=opts)
    res = drain(sv, len(cases))
    makespan = time.perf_counter() - t0
    st = sv.stats()
    sv.close()
    cap = len(cases) / makespan
    rate = 0.8 * cap
    rng = inputs.SplitMix64(77)
    arrivals = np.cumsum([-np.log(1.0 - rng.uniform()) / rate for _ in cases])
    sv = pbfb.Server(budget, max_inflight, cached_meshes=16)
    t0 = time.perf_counter()
    got = []
    for i, c in enumerate(cases):
        while time.perf_counter() - t0 < arrivals[i]:
            got += sv.poll(64, 1000)
        sv.submit(c, i, opts=opts)
    got += drain(sv, len(cases) - len(got))
    span = time.perf_counter() - t0
    st2 = sv.stats()
    sv.close()
    lat = np.array([r["t_done_ms"] - r["t_submit_ms"] for r in got])
    ok = all(r["status"] == 0 for r in res + got)
    energies = {int(r["id"]): r["total"] for r in res}
    tri = {i: int(c.gm_tris.shape[0]) for i, c in enumerate(cases)}
    failed = [{"id": int(r["id"]), "triangles": tri[int(r["id"])], "status": int(r["status"]),
               "error": r["error"][:160]} for r in res + got if r["status"] != 0]
    per_request = [{"id": int(r["id"]), "triangles": tri[int(r["id"])], "latency_ms": round(r["t_done_ms"] - r["t_submit_ms"], 1),
                    "service_ms": round(r["t_done_ms"] - r["t_start_ms"], 1), "newton": int(r["newton_iters"]),
                    "gmres": r["gmres"]} for r in sorted(got, key=lambda r: int(r["id"]))]
    return {"requests": len(cases), "max_inflight": max_inflight, "budget_bytes": budget,
            "saturation_solves_per_s": cap, "peak_bytes": st["peak"],
            "open_loop_rate_per_s": rate, "open_loop_solves_per_s": len(cases) / span,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "all_ok": ok, "resident_mesh_hits": [int(st["mesh_hits"]), int(st2["mesh_hits"])],
            "precision": "fp64" if precision == pbfb.FP64 else "mixed",
            "energies_kcal_mol": [energies[i] for i in sorted(energies)],
            "failed": failed, "per_request": per_request if detail else None,
            "workload": "sphere (1-200 charges) or double helix (8-24 bp) by a fair coin, 2000-8000 "
                        "triangles per surface (log-uniform), 0.01-1 M, eps_in 2 or 4; mixed precision, "
                        "paper tolerances; up to 16 meshes kept resident between requests"}


def run_pbfb(args):
    import numpy as np
    import torch
    import torch.distributed as tdist
    from paper_2511_21713_gb300 import build as pbuild
    pbuild.build()
    from paper_2511_21713_gb300 import inputs, pbfb

    ws, rank, local = dist()
    if ws > 1:
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    case = inputs.multi_charge_sphere() if args.workload == "multi_charge_sphere" else inputs.single_charge_sphere()
    prec = pbfb.MIXED if args.precision == "mixed" else pbfb.FP64
    opts = pbfb.default_opts(precision=prec,
                             residual_update=args.residual_update if prec == pbfb.MIXED else 0.0,
                             residual_far=RESIDUAL_FAR[args.residual_far])
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    mesh = pbfb.Mesh.from_case(case)
    mesh.charges_set(case.q_xyz, case.q_z)
    torch.cuda.synchronize()
    create_ms = 1e3 * (time.perf_counter() - t_setup)
    # launch shapes picked by the autotuner on this mesh (outside the timed region)
    mesh.set_params(case.eps_in, case.eps_out, case.kappa, case.T, prec)
    t_tune = time.perf_counter()
    tuned, tuned_ms = mesh.autotune(reps=3, cache_file=args.tune_cache)
    tune_s = time.perf_counter() - t_tune
    x_out = torch.empty(mesh.n, dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    stream = torch.cuda.current_stream()

    # the first solve also builds what depends on the mesh and kappa only (the Gamma_s
    # near-field corrections and the dense single-layer inverses of the preconditioner);
    # later solves on the same mesh and kappa reuse them
    res = None
    first_ms = None
    mesh.profile(enable=True, reset=True)
    for w in range(args.warmup):
        t0 = time.perf_counter()
        res = mesh.solve_device(case.eps_in, case.eps_out, case.kappa, case.T, x_out, opts)
        torch.cuda.synchronize()
        if w == 0:
            first_ms = 1e3 * (time.perf_counter() - t0)
    setup_prof = mesh.profile(enable=False, reset=True)
    torch.cuda.synchronize()
    if ws > 1:
        tdist.barrier()
    clocks = Clocks(local)
    mesh.profile(enable=True, reset=True)
    clocks.start()
    step_ms = []
    results = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed_step")   # lets a profiler select the timed solves
        e0.record(stream)
        res = mesh.solve_device(case.eps_in, case.eps_out, case.kappa, case.T, x_out, opts)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.nvtx.range_pop()
        step_ms.append(e0.elapsed_time(e1))
        results.append(res)
    torch.cuda.synchronize()
    if ws > 1:
        tdist.barrier()
    clk = clocks.stop()
    prof = mesh.profile(enable=False, reset=True)
    total_ms = sum(step_ms)
    total_ms_max = max_over_ranks(total_ms, dev, ws)

    # end to end through the public C ABI with host buffers: charges in, solution out
    e2e_ms = []
    h2d = case.q_xyz.nbytes + case.q_z.nbytes
    d2h = 8 * mesh.n + 8 * 4
    for _ in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mesh.charges_set(case.q_xyz, case.q_z)
        xh, r2 = mesh.solve(case.eps_in, case.eps_out, case.kappa, case.T, opts)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_val = ws * len(e2e_ms) / (sum(e2e_ms) / 1e3) if e2e_ms else None

    # roofline of the dominant kernel from its live CUDA-event timing (in the timed region): in the
    # mixed precision the float32 far field of the GMRES operator or the float-float far field of
    # the Newton residual, whichever takes the larger share of the step; float64 otherwise.  Work =
    # the method's float32 flops per ordered pair (20 Laplace, 28 Yukawa; the two surfaces have
    # equal point counts here, so 24 per pair on average) x the pairs a launch evaluates; peak =
    # SMs (read from the device) x 128 lanes x 2 flops x the maximum SM clock
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clk.get("sm_max_mhz") or SM_MAX_MHZ
    peak32 = sm_count * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    peak_basis = (f"fp32 non-tensor: {sm_count} SMs (device attribute) x {FP32_LANES} lanes x 2 flops (FMA) x "
                  f"{sm_mhz:.0f} MHz (maximum SM clock) = {peak32:.2f} TFLOP/s; work = "
                  f"{FLOP_PAIR['laplace']:.0f} flops per ordered Laplace pair and {FLOP_PAIR['yukawa']:.0f} per "
                  f"Yukawa pair x the (6 N_t)^2 pairs of each launch")
    fpair = 0.5 * (FLOP_PAIR["laplace"] + FLOP_PAIR["yukawa"])
    cands = []
    if prec == pbfb.MIXED:
        l32, ms32 = prof["nbody_launches"], prof["nbody_ms"]
        if l32:
            tree = tuned.get("treecode") in (2, 3)
            name32 = (f"k_tree_eval + k_tree_up_leaf + k_tree_m2c (float32 far field of the GMRES operator "
                      f"through the treecode: near pairs and cluster proxies, packed, "
                      f"{4 if tuned.get('treecode') == 3 else 2} targets per thread)" if tree
                      else "k_nbody_f32x2 (float32 far field of the GMRES operator, packed, 2 targets per thread)")
            cands.append(dict(kernel=name32, launches=l32, ms=ms32, pairs=prof["nbody_pairs"],
                              flops=prof["nbody_pairs"] * fpair, peak=peak32,
                              traffic=None if tree else NBODY_TRAFFIC,
                              peak_basis=peak_basis))
        lff, msff = prof["nbodyff_launches"], prof["nbodyff_ms"]
        packed_ff = tuned.get("ff_kernel") == 4
        if lff:
            cands.append(dict(kernel="k_nbody_ffm2 (float-float far field of the Newton residual, mutual pairs, "
                                     "2 targets per thread)" if packed_ff else
                                     "k_nbody_ffm (float-float far field of the Newton residual, mutual pairs)",
                              launches=lff, ms=msff, pairs=prof["nbodyff_pairs"],
                              flops=prof["nbodyff_pairs"] * fpair,
                              lane_ops=prof["nbodyff_pairs"] * 0.5 * (FF_OPS_PAIR["laplace"] + FF_OPS_PAIR["yukawa"]),
                              peak=peak32, traffic=FF2_TRAFFIC if packed_ff else FF_TRAFFIC,
                              peak_basis=peak_basis))
    else:
        l64, ms64 = prof["nbody64_launches"], prof["nbody64_ms"]
        cands.append(dict(kernel="k_nbody_f64", launches=l64, ms=ms64, pairs=prof["nbody64_pairs"],
                          flops=prof["nbody64_pairs"] * fpair,
                          peak=1.25, traffic=None, peak_basis="fp64 nominal 1.25 TFLOP/s (GB300)"))

    def roofline_of(c):
        launches = max(c["launches"], 1)
        avg_ms = c["ms"] / launches
        achieved = (c["flops"] / launches) / (avg_ms * 1e-3) / 1e12 if avg_ms > 0 else None
        emu = None
        if c.get("lane_ops") and avg_ms > 0:
            peak_lanes = sm_count * FP32_LANES * sm_mhz * 1e6 / 1e12
            a = (c["lane_ops"] / launches) / (avg_ms * 1e-3) / 1e12
            emu = {"note": "float-float emulation: float32 lane operations issued per ordered pair (ncu) "
                           f"{FF_OPS_PAIR['laplace']} Laplace / {FF_OPS_PAIR['yukawa']} Yukawa against the "
                           "method's 20 / 28 flops",
                   "achieved": a, "peak": peak_lanes, "unit": "T float32 lane-ops/s", "frac": a / peak_lanes}
        return {"bound": "alu", "kernel": c["kernel"], "achieved": achieved, "peak": c["peak"],
                "unit": "TFLOP/s", "frac": (achieved / c["peak"]) if achieved else None,
                "traffic": c["traffic"] if args.workload == "multi_charge_sphere" else None,
                "peak_basis": c["peak_basis"], "avg_launch_ms": avg_ms,
                "pairs_per_launch": c["pairs"] / launches, "launches": c["launches"],
                "share_of_step": c["ms"] / total_ms if total_ms else None,
                "float_float_emulation": emu}

    rooflines = sorted((roofline_of(c) for c in cands), key=lambda r: -(r["share_of_step"] or 0))

    out = {
        "metric": METRIC, "value": job_throughput(ws, args.steps, total_ms_max), "unit": "solves/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec == pbfb.MIXED else "f64",
        "data": "synthetic (seeded sphere mesh and charges)",
        "config": workload_config(case, args.precision) | {"parallelism": f"replicas x{ws}",
                                                            "residual_update": opts.residual_update,
                                                            "residual_far": args.residual_far},
        "p50_ms": statistics.median(step_ms),
        "p99_ms": float(np.percentile(step_ms, 99)),
        "e2e": {"value": e2e_val, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(prof["launches"]),
        "roofline": rooflines[0],
        "roofline_next": rooflines[1] if len(rooflines) > 1 else None,
        "clocks": clk,
        "autotune": {"shapes": tuned, "best_ms": tuned_ms, "seconds": tune_s},
        "setup": {"mesh_create_and_charges_ms": create_ms, "first_solve_ms": first_ms,
                  "dense_single_layer_build_ms": setup_prof["dense_build_ms"],
                  "note": "one-time per mesh (and per kappa for Gamma_s); not in the timed steps"},
        "solve": {"newton_iters": res["newton_iters"], "linear_gmres": res["linear_gmres"],
                  "gmres": res["gmres"], "omega": [round(w, 4) for w in res["omega"]],
                  "total_kcal_mol": res["total"], "LC": res["LC"], "NC": res["NC"], "dG_ion": res["dG_ion"]},
    }
    # the plain float64 GPU path on the same input and mesh: one untimed solve, then as many solves
    # as the mixed arm timed, each with CUDA events after an L2 flush (after the mixed arm's timed
    # region, so that its clock record covers the headline number alone)
    if args.fp64_compare and prec == pbfb.MIXED:
        o64 = pbfb.default_opts(precision=pbfb.FP64)
        n64 = args.steps if args.fp64_steps < 0 else args.fp64_steps
        r64 = mesh.solve_device(case.eps_in, case.eps_out, case.kappa, case.T, x_out, o64)
        ms64 = []
        for _ in range(n64):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r64 = mesh.solve_device(case.eps_in, case.eps_out, case.kappa, case.T, x_out, o64)
            e1.record(stream)
            e1.synchronize()
            ms64.append(e0.elapsed_time(e1))
        if ms64:
            m64 = sum(ms64) / len(ms64)
            out["fp64_gpu"] = {"steps": len(ms64), "warmup": 1, "ms_per_solve": m64,
                               "solves_per_s": len(ms64) / (sum(ms64) / 1e3),
                               "p50_ms": statistics.median(ms64), "p99_ms": float(np.percentile(ms64, 99)),
                               "mixed_speedup": m64 / (total_ms_max / args.steps),
                               "mixed_energy_rel_diff": abs(res["total"] - r64["total"]) / abs(r64["total"]),
                               "newton_iters": r64["newton_iters"], "gmres": r64["gmres"],
                               "total_kcal_mol": r64["total"]}
            if os.path.exists(GOLDEN):
                ref = json.load(open(GOLDEN))["tight"]["total"]
                out["fp64_gpu"]["energy_rel_err_vs_oracle"] = abs(r64["total"] - ref) / abs(ref)
    # the mixed path with the float-float residual evaluated at every Newton step (residual_update = 0)
    if prec == pbfb.MIXED and args.residual_update > 0:
        o0 = pbfb.default_opts(precision=pbfb.MIXED)
        ms0 = []
        for _ in range(max(1, min(args.steps, 5))):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r0 = mesh.solve_device(case.eps_in, case.eps_out, case.kappa, case.T, x_out, o0)
            e1.record(stream)
            e1.synchronize()
            ms0.append(e0.elapsed_time(e1))
        out["mixed_residual_every_step"] = {"steps": len(ms0), "ms_per_solve": sum(ms0) / len(ms0),
                                            "newton_iters": r0["newton_iters"], "total_kcal_mol": r0["total"]}
    # the other far field of the Newton residual's full evaluations (float-float or float32)
    if prec == pbfb.MIXED:
        alt = "f32" if args.residual_far == "float2" else "float2"
        oa = pbfb.default_opts(precision=pbfb.MIXED, residual_update=args.residual_update,
                               residual_far=RESIDUAL_FAR[alt])
        msa = []
        for _ in range(max(1, min(args.steps, 5))):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ra = mesh.solve_device(case.eps_in, case.eps_out, case.kappa, case.T, x_out, oa)
            e1.record(stream)
            e1.synchronize()
            msa.append(e0.elapsed_time(e1))
        out["mixed_residual_far_" + alt] = {"steps": len(msa), "ms_per_solve": sum(msa) / len(msa),
                                            "newton_iters": ra["newton_iters"], "total_kcal_mol": ra["total"],
                                            "energy_rel_diff_vs_headline": abs(ra["total"] - res["total"]) /
                                            abs(res["total"])}
    if args.full_formulation and ws == 1 and args.workload == "multi_charge_sphere":
        out["full_formulation"] = run_full_formulation(pbfb, inputs, tuned, opts, res, flush, stream)
    if args.helix > 0 and ws == 1 and args.workload == "multi_charge_sphere":
        out["double_helix"] = run_helix(pbfb, inputs, opts, flush, stream, args.helix)
    if args.serving > 0 and args.workload == "multi_charge_sphere":
        cases = serving_cases(args.serving)
        out["serving"] = run_serving(pbfb, cases, 4, 64 << 30, args.residual_update,
                                     residual_far=args.residual_far)
    if os.path.exists(GOLDEN) and args.workload == "multi_charge_sphere":
        g = json.load(open(GOLDEN))
        ref = g["tight"]["total"]
        out["energy_rel_err_vs_oracle"] = abs(res["total"] - ref) / abs(ref)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and args.workload == "multi_charge_sphere":
        out["cpu_baseline"] = cpu_baseline(case, args.cpu_sample)
    if ws > 1:
        tdist.destroy_process_group()
    mesh.close()
    return out if rank == 0 else None


def run_full_formulation(pbfb, inputs, shapes, opts, shell_res, flush, stream, steps=3):
    """The paper's own formulation (FEM over Omega_m and Omega_i with the charges as point loads,
    lam_m from the Gamma_m equation afterwards) on the bench sphere meshed inside Gamma_m as well:
    the same surfaces, shell and charges, one warm-up solve, then solves timed with CUDA events."""
    import torch
    case = inputs.multi_charge_solute_sphere()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m = pbfb.Mesh.from_case(case)
    m.charges_set(case.q_xyz, case.q_z)
    torch.cuda.synchronize()
    create_ms = 1e3 * (time.perf_counter() - t0)
    m.apply_tuning(shapes)
    x = torch.empty(m.n, dtype=torch.float64, device="cuda")
    r = m.solve_device(case.eps_in, case.eps_out, case.kappa, case.T, x, opts)
    ms = []
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = m.solve_device(case.eps_in, case.eps_out, case.kappa, case.T, x, opts)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    out = {"workload": case.name, "n_v": m.n_v, "n_t": m.n_t, "n_t_omega_m": int((case.tet_region == 0).sum()),
           "steps": steps, "solves_per_s": steps / (sum(ms) / 1e3), "ms_per_solve": sum(ms) / steps,
           "mesh_create_and_charges_ms": create_ms, "newton_iters": r["newton_iters"], "gmres": r["gmres"],
           "linear_gmres": r["linear_gmres"], "gamma_m_flux_and_energy_ms": r["ms_energy"],
           "total_kcal_mol": r["total"], "LC": r["LC"], "NC": r["NC"], "dG_ion": r["dG_ion"],
           "rel_diff_vs_three_region": abs(r["total"] - shell_res["total"]) / abs(shell_res["total"])}
    m.close()
    return out


def run_helix(pbfb, inputs, opts, flush, stream, steps=2):
    """The synthetic double helix (24 base pairs, 40,500 triangles per surface, 1,944,000 tets,
    1548 charges, 0.15 M; surface potentials above 10 kT/e): mesh creation and charges, one untimed
    solve (it builds the Gamma_s corrections, the dense single-layer inverses and the far-field
    trees), then `steps` solves timed with CUDA events after an L2 flush."""
    import torch
    t0 = time.perf_counter()
    case = inputs.double_helix()
    gen_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m = pbfb.Mesh.from_case(case)
    m.charges_set(case.q_xyz, case.q_z)
    torch.cuda.synchronize()
    create_ms = 1e3 * (time.perf_counter() - t0)
    x = torch.empty(m.n, dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    r = m.solve_device(case.eps_in, case.eps_out, case.kappa, case.T, x, opts)
    torch.cuda.synchronize()
    first_ms = 1e3 * (time.perf_counter() - t0)
    m.profile(enable=True, reset=True)
    ms = []
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = m.solve_device(case.eps_in, case.eps_out, case.kappa, case.T, x, opts)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    prof = m.profile(enable=False, reset=True)
    tot = sum(ms)
    out = {"workload": case.name, "n_v": m.n_v, "n_t": m.n_t, "gamma_m_triangles": int(case.gm_tris.shape[0]),
           "gamma_s_triangles": int(case.gs_tris.shape[0]), "charges": int(len(case.q_z)),
           "net_charge_e": float(case.q_z.sum()), "kappa_per_A": case.kappa, "steps": steps,
           "solves_per_s": steps / (tot / 1e3), "ms_per_solve": tot / steps,
           "input_generation_s": gen_s, "mesh_create_and_charges_ms": create_ms, "first_solve_ms": first_ms,
           "newton_iters": r["newton_iters"], "gmres": r["gmres"], "linear_gmres": r["linear_gmres"],
           "omega": [round(w, 4) for w in r["omega"]], "total_kcal_mol": r["total"], "LC": r["LC"],
           "NC": r["NC"], "dG_ion": r["dG_ion"], "tuning": m.get_tuning(),
           "share_float32_far_field": prof["nbody_ms"] / tot if tot else None,
           "share_float_float_far_field": prof["nbodyff_ms"] / tot if tot else None,
           "float32_pairs_per_launch": prof["nbody_pairs"] / max(prof["nbody_launches"], 1)}
    m.close()
    return out


def _mixed_case(seed, kw):
    sys.path.insert(0, ROOT)
    from paper_2511_21713_gb300 import inputs
    return inputs.mixed_case(seed, **kw)


def generate_cases(seeds, **kw):
    """Instances of inputs.mixed_case, generated in a pool of freshly spawned host processes."""
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(max(1, min(len(seeds), os.cpu_count() or 1))) as pool:
        return pool.starmap(_mixed_case, [(sd, kw) for sd in seeds])


def run_batch(args):
    """Many uneven instances solved concurrently (pbfb_solve_batch: host threads, one CUDA stream per
    mesh, every instance's work overlapping on the GPU): spheres of 2000-8000 triangles and 1-200
    charges, double helices of 8-48 base pairs on 5000-40000 triangles, at most 2M tets, 0.01-1 M,
    mixed precision; launch shapes from the autotuner (cached per size bucket).  One untimed batch
    (it builds what depends on the mesh and kappa), then `steps` timed batches.  Each instance's
    result is checked against its own single solve on a few instances (bitwise)."""
    import numpy as np
    import torch
    cases = generate_cases(list(range(4000, 4000 + args.instances)))
    from paper_2511_21713_gb300 import build as pbuild
    pbuild.build()
    from paper_2511_21713_gb300 import pbfb
    opts = pbfb.default_opts(precision=pbfb.MIXED, residual_update=args.residual_update,
                             residual_far=RESIDUAL_FAR[args.residual_far])
    streams = [torch.cuda.Stream() for _ in cases]
    t0 = time.perf_counter()
    meshes = []
    for c, st in zip(cases, streams):
        m = pbfb.Mesh.from_case(c, stream=st.cuda_stream)
        m.charges_set(c.q_xyz, c.q_z)
        meshes.append(m)
    create_s = time.perf_counter() - t0
    cache = os.path.join(tempfile.mkdtemp(), "tune.json")
    t0 = time.perf_counter()
    for c, m in zip(cases, meshes):
        m.set_params(c.eps_in, c.eps_out, c.kappa, c.T, pbfb.MIXED)
        m.autotune(reps=1, cache_file=cache)
    tune_s = time.perf_counter() - t0
    params = [(c.eps_in, c.eps_out, c.kappa, c.T, opts) for c in cases]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    first = pbfb.solve_batch(meshes, params, max_concurrent=args.concurrency)
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    clocks = Clocks(0)
    clocks.start()
    walls = []
    res = None
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = pbfb.solve_batch(meshes, params, max_concurrent=args.concurrency)
        torch.cuda.synchronize()
        walls.append(time.perf_counter() - t0)
    clk = clocks.stop()
    same = []
    for i in range(0, len(cases), max(1, len(cases) // 4)):
        c = cases[i]
        r1 = meshes[i].solve_device(c.eps_in, c.eps_out, c.kappa, c.T, None, opts)
        same.append(r1["total"] == res[i]["total"] and r1["gmres"] == res[i]["gmres"])
    tris = np.array([c.gm_tris.shape[0] for c in cases])
    tets = np.array([c.n_t for c in cases])
    out = {"metric": METRIC, "config": {"workload": "batch of uneven instances",
                                        "instances": len(cases), "helices": int(sum("helix" in c.name for c in cases)),
                                        "triangles_per_surface": [int(tris.min()), int(np.median(tris)), int(tris.max())],
                                        "tets": [int(tets.min()), int(np.median(tets)), int(tets.max())],
                                        "max_concurrent": args.concurrency, "precision": "mixed",
                                        "residual_update": opts.residual_update,
                                        "note": "instances overlap through host threads and one CUDA stream per "
                                                "mesh (pbfb_solve_batch), not one persistent launch"},
           "value": len(cases) * len(walls) / sum(walls), "unit": "solves/s", "steps": len(walls),
           "batch_wall_s": walls, "first_batch_s": first_s, "mesh_create_s": create_s, "autotune_s": tune_s,
           "newton_iters": [r["newton_iters"] for r in res], "all_ok": all(r["status"] == 0 for r in res),
           "alone_equals_batched": same, "clocks": clk}
    for m in meshes:
        m.close()
    return out


def run_serving_config(args):
    """Serving at the configuration's sizes: a seeded Poisson-arrival stream of `requests` solves,
    spheres or double helices by a fair coin, 2000-80000 surface triangles (log-uniform; at most 2M
    tets), eps_in 2 or 4, 0.01-1 M; admitted by HBM budget, solved concurrently with resident
    meshes.  Mixed arm: saturation capacity, then arrivals at 0.8x capacity (p50 / p99 from arrival to
    result).  Float64 arm: the same for the requests of at most `fp64_max_tri` triangles (the float64
    far field makes larger surfaces take minutes), on the same stream order."""
    import numpy as np
    import torch
    cases = generate_cases(list(range(5000, 5000 + args.requests)), sphere_tri=(2000.0, 80000.0),
                           helix_tri=(2000.0, 80000.0))
    from paper_2511_21713_gb300 import build as pbuild
    pbuild.build()
    from paper_2511_21713_gb300 import pbfb
    torch.cuda.init()
    tris = np.array([c.gm_tris.shape[0] for c in cases])
    out = {"metric": METRIC, "config": {"workload": "serving stream", "requests": len(cases),
                                        "triangles_per_surface": [int(tris.min()), int(np.median(tris)),
                                                                  int(tris.max())],
                                        "helices": int(sum("helix" in c.name for c in cases)),
                                        "budget_bytes": args.budget_gb << 30, "max_inflight": args.concurrency,
                                        "residual_update": args.residual_update,
                                        "residual_far": args.residual_far}}
    out["mixed"] = run_serving(pbfb, cases, args.concurrency, args.budget_gb << 30, args.residual_update,
                               detail=True, residual_far=args.residual_far)
    small = [c for c in cases if c.gm_tris.shape[0] <= args.fp64_max_tri]
    if small and args.fp64_max_tri > 0:
        out["fp64"] = run_serving(pbfb, small, args.concurrency, args.budget_gb << 30, 0.0, precision=pbfb.FP64)
        out["mixed_same_subset"] = run_serving(pbfb, small, args.concurrency, args.budget_gb << 30,
                                               args.residual_update, residual_far=args.residual_far)
        # every request of the subset checked against the float64 GPU path (itself checked against
        # the oracle at full size): the metric's bound is 1e-5 relative on the energy
        e64 = np.array(out["fp64"]["energies_kcal_mol"])
        emx = np.array(out["mixed_same_subset"]["energies_kcal_mol"])
        err = np.abs(emx - e64) / np.abs(e64)
        out["mixed_vs_fp64_energy_rel_err"] = {"max": float(err.max()), "median": float(np.median(err)),
                                               "requests": int(err.size), "within_1e-5": bool(err.max() <= 1e-5)}
    return out


def oracle_counts():
    """Work counts of the oracle's own solve of the bench workload at the paper's tolerances
    (tests/golden/multi_charge_sphere.json, written by the oracle alone): Newton steps,
    operator applications (GMRES iterations, one true residual per restart cycle, one residual
    c and one search direction p per Newton step) and batched omega evaluations."""
    import math
    g = json.load(open(GOLDEN))
    d = g["default"]
    k = d["newton_iters"]
    cyc = lambda its: max(1, math.ceil(its / 200))
    applies = d["linear_gmres"] + cyc(d["linear_gmres"])
    applies += sum(its + cyc(its) + 1 for its in d["gmres"])
    applies += sum(1 for ev in d["omega_evals"] if ev > 0)
    return {"newton_iters": k, "assemblies": k + 1, "applies": applies, "omega_evals": sum(d["omega_evals"]),
            "measured_setup_s": g["setup_s"], "measured_solve_s": d["seconds"]}


def oracle_sample(case, counts, frac_rows):
    """Time the oracle on a bounded sample of the workload and scale it to one solve.

    Sample: dense Galerkin BEM assembly of 1/frac_rows of the test triangles of each surface
    (both operators, all quadrature classes), the sparse FEM set-up and Coulomb data, one
    nonlinear load + Jacobian assembly over all tets, one omega evaluation, one coupled dense
    apply and one energy evaluation.  One solve is modelled as set-up + frac_rows x the BEM
    sample + assemblies x assembly + omega evaluations x evaluation + applies x apply + energy,
    with the oracle's own counts (oracle_counts).
    """
    import numpy as np
    import scipy.sparse as sp
    from oracle import bem, fem, pb
    t = {}
    t0 = time.perf_counter()
    P = object.__new__(pb.Problem)
    # the problem's pieces without the full dense assembly
    P.case = case
    P.eps_m, P.eps_s, P.kappa, P.T = case.eps_in, case.eps_out, case.kappa, case.T
    P.kT = pb.KB * P.T
    P.lB = pb.COULOMB / P.kT
    P.coef = P.eps_s * P.kappa ** 2
    P.xyz, P.tets, P.nv = case.xyz, case.tets, case.xyz.shape[0]
    P.sm, P.ss = bem.Surface(case.xyz, case.gm_tris), bem.Surface(case.xyz, case.gs_tris)
    P.nm, P.ns = P.sm.n, P.ss.n
    P.n = P.nv + P.nm + P.ns
    P.A = fem.stiffness(case.xyz, case.tets, P.eps_s)
    P.Mm, P.Ms = bem.mass_matrix(P.sm), bem.mass_matrix(P.ss)
    P.Rm = sp.csr_matrix((np.ones(P.nm), (np.arange(P.nm), P.sm.verts)), shape=(P.nm, P.nv))
    P.Rs = sp.csr_matrix((np.ones(P.ns), (np.arange(P.ns), P.ss.verts)), shape=(P.ns, P.nv))
    P.B_um = P.eps_m * (P.Rm.T @ P.Mm)
    P.B_us = -P.eps_s * (P.Rs.T @ P.Ms)
    P.b = np.zeros(P.n)
    P.b[P.nv:P.nv + P.nm] = (P.lB / P.eps_m) * bem.coulomb_rhs(P.sm, case.q_xyz, case.q_z)
    t["setup_fem_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    sub_m = np.arange(0, P.sm.nt, frac_rows)
    sub_s = np.arange(0, P.ss.nt, frac_rows)
    # dense matrices of the full size with the sampled rows filled: the apply below costs what it
    # costs on the complete matrices
    P.VL, P.KL = bem.assemble(P.sm, 0.0, test_tris=sub_m)
    P.VY, P.KY = bem.assemble(P.ss, P.kappa, test_tris=sub_s)
    t["bem_sample_s"] = time.perf_counter() - t0
    u = np.zeros(P.nv) + 0.5
    t0 = time.perf_counter()
    P.N(u, "HS")
    Jm = P.J(u, "HS")
    t["assembly_s"] = time.perf_counter() - t0
    x = np.ones(P.n)
    t0 = time.perf_counter()
    P.apply(x, Jm)
    t["apply_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    pb.omega_dots(P, u, u, np.ones(P.n), np.ones(P.n), 1.0, "HS")
    t["omega_eval_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    pb.energy(P, x, x)
    t["energy_s"] = time.perf_counter() - t0
    sample_s = sum(t.values())
    model_s = (t["setup_fem_s"] + frac_rows * t["bem_sample_s"] + counts["assemblies"] * t["assembly_s"]
               + counts["omega_evals"] * t["omega_eval_s"] + counts["applies"] * t["apply_s"] + t["energy_s"])
    return {"model_s_per_solve": model_s, "sample_s": sample_s, "parts_s": {kk: round(v, 4) for kk, v in t.items()},
            "description": (f"oracle (numpy float64) on this workload: BEM assembly of 1/{frac_rows} of the test "
                            f"triangles per surface, FEM set-up and Coulomb data, one load+Jacobian assembly, one "
                            f"omega evaluation, one dense coupled apply, one energy ({sample_s:.1f} s measured); one "
                            f"solve modelled with the oracle's own counts ({counts['assemblies']} assemblies, "
                            f"{counts['omega_evals']} omega evaluations, {counts['applies']} applies) = "
                            f"{model_s:.1f} s")}


# a complete oracle solve of the small single-charge sphere (radius 4, shell to 10, nu = 5,
# 13 layers, +5 e), run in a fresh interpreter so that its thread limits apply from the start
_ORACLE_FULL = r"""
import json, sys, time
sys.path.insert(0, sys.argv[1])
from paper_2511_21713_gb300 import inputs
from oracle import pb
case = inputs.single_charge_sphere()
t0 = time.perf_counter()
P = pb.Problem(case)
t1 = time.perf_counter()
R = pb.solve(P, pb.Opts())
t2 = time.perf_counter()
print(json.dumps(dict(setup_s=t1 - t0, solve_s=t2 - t1, total_s=t2 - t0, newton_iters=R.newton_iters,
                      total=R.total)))
"""


def oracle_full_solve(threads):
    """Wall time of one complete oracle solve (set-up and solve) of the single-charge sphere with
    BLAS/OpenMP limited to `threads`."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = str(threads)
    r = subprocess.run([sys.executable, "-c", _ORACLE_FULL, ROOT], env=env, capture_output=True, text=True,
                       timeout=900)
    if r.returncode != 0:
        return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else f"rc {r.returncode}"}
    return json.loads(r.stdout.strip().splitlines()[-1]) | {"threads": threads}


def cpu_baseline(case, frac_rows):
    """The oracle timed on this host: the bench workload by the sampled model (value), and complete
    solves of the single-charge sphere with one thread and with every core."""
    counts = oracle_counts()
    smp = oracle_sample(case, counts, frac_rows)
    cores = os.cpu_count() or 1
    full = {"workload": "single_charge_sphere (3528 vertices, 19,500 tets, 500 + 500 triangles, +5 e)",
            "one_thread": oracle_full_solve(1), "all_cores": oracle_full_solve(cores)}
    return {"value": 1.0 / smp["model_s_per_solve"], "unit": "solves/s", "cores": cores, "kind": "oracle",
            "estimate": "model",
            "sample": smp["description"],
            "parts_s": smp["parts_s"], "model_s_per_solve": smp["model_s_per_solve"],
            "model_check": (f"the same model on the host that ran the oracle's complete solve of this workload "
                            f"({ORACLE_C2_MEASURED_HOST}: {counts['measured_setup_s']:.0f} s set-up + "
                            f"{counts['measured_solve_s']:.0f} s solve) predicted "
                            f"{ORACLE_C2_MODEL_ON_THAT_HOST:.0f} s"),
            "measured_full_solves": full}


def run_reference(args):
    """The CPU oracle arm: each step is a bounded oracle sample of the workload (its real duration
    is the step time); the value is solves/s of the modelled complete solve."""
    from paper_2511_21713_gb300 import inputs
    ws, rank, _ = dist()
    if rank != 0:
        return None
    case = inputs.multi_charge_sphere()
    counts = oracle_counts()
    for _ in range(args.warmup):
        pass  # the oracle keeps no state between samples: nothing to warm up
    models, samples = [], []
    last = None
    for _ in range(args.steps):
        last = oracle_sample(case, counts, args.ref_sample)
        models.append(last["model_s_per_solve"])
        samples.append(last["sample_s"])
    v = len(models) / sum(models)
    cores = os.cpu_count() or 1
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(samples) / len(samples),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded sphere mesh and charges)",
            "config": workload_config(case, "fp64 (CPU oracle)") | {
                "parallelism": "1 host process",
                "preconditioner": "Jacobi (the oracle's GMRES: diagonal of the coupled operator)",
                "residual": "float64 at every Newton step"},
            "step": "one bounded sample of the workload (see cpu_baseline.sample); ms_per_step is its measured "
                    "duration, value the modelled complete solve's rate",
            "model_s_per_solve": sum(models) / len(models),
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": cores, "kind": "oracle", "estimate": "model",
                             "sample": last["description"]},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_step(args):
    """One step of the solve, repeated, for focused profiler captures (-k on the kernel of
    interest): farfield_f32 / farfield_ff / farfield_f64 (V then K on Gamma_m and Gamma_s),
    assemble (sinh Jacobian + load), omega (batched evaluation, 16 values), gmres (one
    block-preconditioned GMRES solve at 1e-6).  Prints the wall time of each repetition."""
    import numpy as np
    import torch
    from paper_2511_21713_gb300 import build as pbuild
    pbuild.build()
    from paper_2511_21713_gb300 import inputs, pbfb
    case = inputs.multi_charge_sphere() if args.workload == "multi_charge_sphere" else inputs.single_charge_sphere()
    m = pbfb.Mesh.from_case(case)
    m.charges_set(case.q_xyz, case.q_z)
    prec = {"farfield_f32": pbfb.MIXED, "farfield_ff": pbfb.FLOAT2, "farfield_f64": pbfb.FP64}.get(args.step,
                                                                                                   pbfb.MIXED)
    m.set_params(case.eps_in, case.eps_out, case.kappa, case.T, prec)
    if args.treecode:
        m.apply_tuning(dict(m.get_tuning(), treecode=args.treecode))
    dev = torch.device("cuda")
    r = np.linalg.norm(case.xyz, axis=1)
    u = torch.as_tensor(4.0 * np.exp(-0.2 * (r - r.min())), device=dev)
    for rep in range(args.reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if args.step.startswith("farfield"):
            for which, n in ((pbfb.GAMMA_M, m.n_m), (pbfb.GAMMA_S, m.n_s)):
                x = torch.ones(n, dtype=torch.float64, device=dev)
                y = torch.zeros_like(x)
                m.bem_apply(which, 0, x, y)
                m.bem_apply(which, 1, x, y)
        elif args.step == "assemble":
            N = torch.zeros(m.n_v, dtype=torch.float64, device=dev)
            m.assemble(pbfb.HS, u, N)
        elif args.step == "omega":
            c = torch.ones(m.n, dtype=torch.float64, device=dev)
            m.omega_eval(pbfb.HS, u, 0.1 * u, c, c, np.linspace(0.25, 4.0, 16))
        elif args.step == "gmres":
            m.assemble(pbfb.HS, u)
            b = torch.ones(m.n, dtype=torch.float64, device=dev)
            x = torch.zeros_like(b)
            m.gmres(b, x, 1e-6, precond=pbfb.BLOCK, inner_iters=30)
        else:
            raise SystemExit(f"unknown step {args.step}")
        torch.cuda.synchronize()
        print(f"{args.step} rep {rep}: {1e3 * (time.perf_counter() - t0):.2f} ms", flush=True)
    m.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pbfb", choices=["pbfb", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--cpu-sample", type=int, default=128, help="1/k of the BEM rows in the oracle sample")
    ap.add_argument("--ref-sample", type=int, default=512,
                    help="1/k of the BEM rows in each step of the reference (oracle) arm")
    ap.add_argument("--step", default=None, help="time one step of the solve (profiling); see run_step")
    ap.add_argument("--reps", type=int, default=2, help="repetitions of --step")
    ap.add_argument("--treecode", type=int, default=0,
                    help="--step farfield_f32: 1 direct sum, 2 treecode (0 built-in)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3, help="host-buffer solves timed for the e2e figure")
    ap.add_argument("--serving", type=int, default=24, help="requests in the serving run (0 = skip)")
    ap.add_argument("--no-fp64-compare", dest="fp64_compare", action="store_false",
                    help="skip the float64-path solves reported under fp64_gpu")
    ap.add_argument("--fp64-steps", type=int, default=-1,
                    help="float64-path solves timed for fp64_gpu (default: as many as --steps)")
    ap.add_argument("--helix", type=int, default=2, help="timed solves of the double helix (0 = skip)")
    ap.add_argument("--config", default="headline", choices=["headline", "batch", "serving"],
                    help="batch: many uneven instances at once; serving: the request stream at 2k-80k triangles")
    ap.add_argument("--instances", type=int, default=64, help="--config batch: instances")
    ap.add_argument("--concurrency", type=int, default=8, help="--config batch/serving: solves in flight")
    ap.add_argument("--requests", type=int, default=64, help="--config serving: requests")
    ap.add_argument("--budget-gb", type=int, default=160, help="--config serving: HBM budget")
    ap.add_argument("--fp64-max-tri", type=int, default=8000,
                    help="--config serving: largest surface (triangles) of the float64 arm")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON file of autotuned shapes (read if it holds this GPU and size bucket, else "
                         "written): a profiling run under ncu then uses the shapes of the plain run")
    ap.add_argument("--residual-far", default="f32", choices=["float2", "f32"],
                    help="far field of the Newton residual's full evaluations (pbfb_newton_opts.residual_far)")
    ap.add_argument("--residual-update", type=float, default=0.5,
                    help="mixed path: pbfb_newton_opts.residual_update (0 = float-float residual every step)")
    ap.add_argument("--no-full-formulation", dest="full_formulation", action="store_false",
                    help="skip the solves of the formulation with Omega_m meshed (full_formulation)")
    ap.add_argument("--workload", default="multi_charge_sphere", choices=["multi_charge_sphere", "small"],
                    help="small = the single-charge sphere, for profiler launch lists")
    args = ap.parse_args()
    if args.step:
        run_step(args)
        return
    if args.config in ("batch", "serving"):
        print(json.dumps(run_batch(args) if args.config == "batch" else run_serving_config(args)))
        return
    out = run_reference(args) if args.impl == "reference" else run_pbfb(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
