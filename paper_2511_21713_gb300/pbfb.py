"""Python binding of libpbfb (include/pbfb.h): argument marshalling only.

Every function here calls the C ABI of the same name; all computation happens in
the CUDA library.  Device buffers are torch CUDA tensors (float64, contiguous);
host buffers are numpy arrays.  Loading fails loudly when libpbfb.so has not
been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpbfb.so")

PBFB_OK = 0
ERRORS = {1: "INVALID", 2: "CUDA", 3: "GMRES_NOCONV", 4: "NEWTON_NOCONV", 5: "OMEGA",
          6: "NONFINITE", 7: "OOM", 8: "STATE", 9: "TIMEOUT"}
ERR_TIMEOUT = 9
FP64, MIXED, FLOAT2 = 0, 1, 2
LINEAR, T3, HS, T5, T7 = 0, 1, 2, 3, 4
NEWTON, PICARD = 0, 1
GAMMA_M, GAMMA_S = 0, 1
JACOBI, BLOCK, BLOCK_DENSE = 0, 1, 2
MAX_TRACE = 64

# every symbol include/pbfb.h declares
EXPORTS = [
    "pbfb_default_opts", "pbfb_mesh_create", "pbfb_mesh_sizes", "pbfb_surface_vertices",
    "pbfb_charges_set", "pbfb_solve", "pbfb_solve_device", "pbfb_mesh_destroy",
    "pbfb_last_error", "pbfb_set_params", "pbfb_assemble", "pbfb_clear_jacobian",
    "pbfb_apply", "pbfb_bem_apply", "pbfb_fem_rows", "pbfb_gmres", "pbfb_omega_eval",
    "pbfb_energy", "pbfb_profile", "pbfb_bem_apply_noalloc", "pbfb_set_tuning",
    "pbfb_server_create", "pbfb_server_submit", "pbfb_server_poll", "pbfb_server_stats",
    "pbfb_server_destroy", "pbfb_solve_batch", "pbfb_single_layer_dense",
    "pbfb_get_tuning", "pbfb_apply_tuning", "pbfb_autotune", "pbfb_mesh_create_full",
    "pbfb_gamma_m_flux", "pbfb_check_charges",
]


class PbfbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pbfb error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class NewtonOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol_nl", ctypes.c_double),
                ("tol_gmres", ctypes.c_double), ("tol_gmres0", ctypes.c_double),
                ("tol_omega", ctypes.c_double), ("L_e", ctypes.c_double),
                ("omega0_first", ctypes.c_double), ("omega0_rest", ctypes.c_double),
                ("omega_max", ctypes.c_double), ("max_newton", ctypes.c_int),
                ("max_gmres", ctypes.c_int), ("restart", ctypes.c_int),
                ("max_omega_iters", ctypes.c_int), ("n_taylor", ctypes.c_int),
                ("taylor", ctypes.c_int * 4), ("method", ctypes.c_int), ("R_e", ctypes.c_double),
                ("omega_warm_start", ctypes.c_int),
                ("omega_search", ctypes.c_int), ("precond", ctypes.c_int),
                ("inner_iters", ctypes.c_int), ("accept_ratio", ctypes.c_double),
                ("residual_update", ctypes.c_double), ("residual_far", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("dG_total", ctypes.c_double), ("dG_LC", ctypes.c_double),
                ("dG_NC", ctypes.c_double), ("dG_Omega_i", ctypes.c_double),
                ("status", ctypes.c_int), ("newton_iters", ctypes.c_int),
                ("linear_gmres_iters", ctypes.c_int), ("omega_fallbacks", ctypes.c_int),
                ("gmres_iters", ctypes.c_int * MAX_TRACE), ("omega", ctypes.c_double * MAX_TRACE),
                ("e", ctypes.c_double * MAX_TRACE), ("omega_evals", ctypes.c_int * MAX_TRACE),
                ("ms_linear", ctypes.c_double), ("ms_newton", ctypes.c_double),
                ("ms_energy", ctypes.c_double), ("residual_updates", ctypes.c_int)]

    def as_dict(self):
        k = self.newton_iters
        return dict(total=self.dG_total, LC=self.dG_LC, NC=self.dG_NC, dG_ion=self.dG_Omega_i,
                    status=self.status, newton_iters=k, linear_gmres=self.linear_gmres_iters,
                    gmres=list(self.gmres_iters[:k]), omega=list(self.omega[:k]), e=list(self.e[:k]),
                    omega_evals=list(self.omega_evals[:k]), omega_fallbacks=self.omega_fallbacks,
                    ms_linear=self.ms_linear, ms_newton=self.ms_newton, ms_energy=self.ms_energy,
                    residual_updates=self.residual_updates)


class Request(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("xyz", ctypes.c_void_p), ("n_v", ctypes.c_int32),
                ("tets", ctypes.c_void_p), ("n_t", ctypes.c_int64), ("gm_tris", ctypes.c_void_p),
                ("n_gm", ctypes.c_int32), ("gs_tris", ctypes.c_void_p), ("n_gs", ctypes.c_int32),
                ("q_xyz", ctypes.c_void_p), ("q_z", ctypes.c_void_p), ("n_q", ctypes.c_int32),
                ("eps_in", ctypes.c_double), ("eps_out", ctypes.c_double), ("kappa", ctypes.c_double),
                ("T", ctypes.c_double), ("opts", ctypes.POINTER(NewtonOpts)), ("tet_region", ctypes.c_void_p)]


class Response(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int), ("result", Result),
                ("t_submit_ms", ctypes.c_double), ("t_start_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double), ("error", ctypes.c_char * 256)]

    def as_dict(self):
        d = self.result.as_dict()
        d.update(id=self.id, status=self.status, t_submit_ms=self.t_submit_ms, t_start_ms=self.t_start_ms,
                 t_done_ms=self.t_done_ms, error=self.error.decode())
        return d


class Tuning(ctypes.Structure):
    _fields_ = [("nbody_targets_per_thread", ctypes.c_int32), ("nbody_blocks_per_sm", ctypes.c_int32),
                ("nbody_packed", ctypes.c_int32), ("ff_blocks_per_sm", ctypes.c_int32),
                ("ff_kernel", ctypes.c_int32), ("spmv_lanes", ctypes.c_int32),
                ("spmv_block", ctypes.c_int32), ("pcg_blocks_per_sm", ctypes.c_int32),
                ("pcg_lanes", ctypes.c_int32), ("treecode", ctypes.c_int32),
                ("pcg_precision", ctypes.c_int32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


class BatchParams(ctypes.Structure):
    _fields_ = [("eps_in", ctypes.c_double), ("eps_out", ctypes.c_double), ("kappa", ctypes.c_double),
                ("T", ctypes.c_double), ("opts", ctypes.POINTER(NewtonOpts))]


_lib = None


def load():
    """Load libpbfb.so (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, D, I, I64, U = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    sig = {
        "pbfb_default_opts": (None, [ctypes.POINTER(NewtonOpts)]),
        "pbfb_mesh_create": (I, [P, I, P, I64, P, I, P, I, U, ctypes.POINTER(P)]),
        "pbfb_mesh_create_full": (I, [P, I, P, I64, P, P, I, P, I, U, ctypes.POINTER(P)]),
        "pbfb_gamma_m_flux": (I, [P, P, I, P]),
        "pbfb_mesh_sizes": (I, [P, P]),
        "pbfb_surface_vertices": (I, [P, I, P]),
        "pbfb_charges_set": (I, [P, P, P, I]),
        "pbfb_check_charges": (I, [P, I, P, I, P, I, P]),
        "pbfb_solve": (I, [P, D, D, D, D, P, P, P, P, P]),
        "pbfb_solve_device": (I, [P, D, D, D, D, P, P, P]),
        "pbfb_mesh_destroy": (I, [P]),
        "pbfb_last_error": (ctypes.c_char_p, []),
        "pbfb_set_params": (I, [P, D, D, D, D, I]),
        "pbfb_assemble": (I, [P, I, P, P]),
        "pbfb_clear_jacobian": (I, [P]),
        "pbfb_apply": (I, [P, P, P]),
        "pbfb_bem_apply": (I, [P, I, I, P, P]),
        "pbfb_bem_apply_noalloc": (I, [P, I, I, P, P]),
        "pbfb_fem_rows": (I, [P, P, P, P]),
        "pbfb_gmres": (I, [P, P, P, D, I, I, I, I, P, P]),
        "pbfb_omega_eval": (I, [P, I, P, P, P, P, P, I, P]),
        "pbfb_energy": (I, [P, P, P, P]),
        "pbfb_profile": (I, [P, I, I, P]),
        "pbfb_set_tuning": (I, [P, I, I, I]),
        "pbfb_server_create": (I, [I, ctypes.c_uint64, I, I, ctypes.POINTER(P)]),
        "pbfb_server_submit": (I, [P, ctypes.POINTER(Request)]),
        "pbfb_server_poll": (I, [P, P, I, I, ctypes.POINTER(ctypes.c_int)]),
        "pbfb_server_stats": (I, [P, P]),
        "pbfb_server_destroy": (I, [P]),
        "pbfb_solve_batch": (I, [P, P, I, I, P]),
        "pbfb_single_layer_dense": (I, [P, I, I, P, ctypes.c_int32]),
        "pbfb_get_tuning": (I, [P, ctypes.POINTER(Tuning)]),
        "pbfb_apply_tuning": (I, [P, ctypes.POINTER(Tuning)]),
        "pbfb_autotune": (I, [P, I, ctypes.POINTER(Tuning), P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(code):
    if code != PBFB_OK:
        raise PbfbError(code, load().pbfb_last_error().decode())


def _ptr(a):
    """Address of a numpy array or a torch tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def default_opts(**kw) -> NewtonOpts:
    o = NewtonOpts()
    load().pbfb_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        if k == "taylor":
            v = list(v)
            o.n_taylor = len(v)
            v = (ctypes.c_int * 4)(*(v + [0] * (4 - len(v))))
        setattr(o, k, v)
    return o


def check_charges(xyz, gm_tris, q_xyz):
    """Winding numbers of Gamma_m at the charges (pbfb_check_charges, host only); raises
    PbfbError (INVALID) when a charge is not strictly inside.  Returns the winding numbers."""
    x = np.ascontiguousarray(xyz, np.float64)
    t = np.ascontiguousarray(gm_tris, np.int32)
    q = np.ascontiguousarray(q_xyz, np.float64).reshape(-1, 3)
    w = np.zeros(q.shape[0])
    _check(load().pbfb_check_charges(_ptr(x), x.shape[0], _ptr(t), t.shape[0], _ptr(q), q.shape[0], _ptr(w)))
    return w


def current_stream() -> int:
    import torch
    return torch.cuda.current_stream().cuda_stream


class Mesh:
    """Owner of a pbfb_mesh handle."""

    def __init__(self, xyz, tets, gm_tris, gs_tris, stream=None, tet_region=None):
        """tet_region None: a shell mesh of Omega_i (pbfb_mesh_create); else per tet 0 (Omega_m)
        or 1 (Omega_i), the mesh of both regions (pbfb_mesh_create_full)."""
        L = load()
        self._keep = [np.ascontiguousarray(xyz, np.float64), np.ascontiguousarray(tets, np.int32),
                      np.ascontiguousarray(gm_tris, np.int32), np.ascontiguousarray(gs_tris, np.int32)]
        x, t, gm, gs = self._keep
        h = ctypes.c_void_p()
        s = current_stream() if stream is None else stream
        self.full = tet_region is not None
        if self.full:
            reg = np.ascontiguousarray(tet_region, np.int32)
            self._keep.append(reg)
            _check(L.pbfb_mesh_create_full(_ptr(x), x.shape[0], _ptr(t), t.shape[0], _ptr(reg), _ptr(gm),
                                           gm.shape[0], _ptr(gs), gs.shape[0], s, ctypes.byref(h)))
        else:
            _check(L.pbfb_mesh_create(_ptr(x), x.shape[0], _ptr(t), t.shape[0], _ptr(gm), gm.shape[0],
                                      _ptr(gs), gs.shape[0], s, ctypes.byref(h)))
        self.h = h
        sz = np.zeros(8, np.int64)
        _check(L.pbfb_mesh_sizes(self.h, _ptr(sz)))
        self.n_v, self.n_t, self.n_m, self.n_s, self.n, self.fem_nnz, self.nnz_m, self.nnz_s = map(int, sz)

    @classmethod
    def from_case(cls, case, stream=None):
        return cls(case.xyz, case.tets, case.gm_tris, case.gs_tris, stream,
                   tet_region=getattr(case, "tet_region", None))

    def surface_vertices(self, which):
        out = np.zeros(self.n_m if which == GAMMA_M else self.n_s, np.int32)
        _check(load().pbfb_surface_vertices(self.h, which, _ptr(out)))
        return out

    def charges_set(self, xyz, z):
        xyz = np.ascontiguousarray(xyz, np.float64)
        z = np.ascontiguousarray(z, np.float64)
        _check(load().pbfb_charges_set(self.h, _ptr(xyz), _ptr(z), int(z.shape[0])))

    def solve(self, eps_in, eps_out, kappa, T, opts=None, outputs=True):
        """Host-buffer solve; returns (x = [u; lam_m; lam_s] numpy or None, result dict)."""
        res = Result()
        if outputs:
            u, lm, ls = np.zeros(self.n_v), np.zeros(self.n_m), np.zeros(self.n_s)
            args = (_ptr(u), _ptr(lm), _ptr(ls))
        else:
            args = (None, None, None)
        code = load().pbfb_solve(self.h, eps_in, eps_out, kappa, T,
                                 ctypes.byref(opts) if opts is not None else None, *args,
                                 ctypes.byref(res))
        _check(code)
        x = np.concatenate([u, lm, ls]) if outputs else None
        return x, res.as_dict()

    def solve_device(self, eps_in, eps_out, kappa, T, x_out=None, opts=None):
        res = Result()
        _check(load().pbfb_solve_device(self.h, eps_in, eps_out, kappa, T,
                                        ctypes.byref(opts) if opts is not None else None,
                                        _ptr(x_out), ctypes.byref(res)))
        return res.as_dict()

    def set_params(self, eps_in, eps_out, kappa, T, precision=FP64):
        _check(load().pbfb_set_params(self.h, eps_in, eps_out, kappa, T, precision))

    def assemble(self, scheme, u_dev, N_out_dev=None):
        _check(load().pbfb_assemble(self.h, scheme, _ptr(u_dev), _ptr(N_out_dev)))

    def clear_jacobian(self):
        _check(load().pbfb_clear_jacobian(self.h))

    def apply(self, x_dev, y_dev):
        _check(load().pbfb_apply(self.h, _ptr(x_dev), _ptr(y_dev)))

    def bem_apply(self, which, op, x_dev, y_dev):
        _check(load().pbfb_bem_apply(self.h, which, op, _ptr(x_dev), _ptr(y_dev)))

    def gamma_m_flux(self, x_dev, coulomb, lam_dev):
        """lam_m from the trace of u on Gamma_m (pbfb_gamma_m_flux); x_dev n-long, lam_dev n_m."""
        _check(load().pbfb_gamma_m_flux(self.h, _ptr(x_dev), int(coulomb), _ptr(lam_dev)))

    def bem_apply_noalloc(self, which, op, x_dev, y_dev):
        """pbfb_bem_apply with its working memory in the library's fixed device array
        (no allocation; at most 65,536 quadrature points per surface)."""
        _check(load().pbfb_bem_apply_noalloc(self.h, which, op, _ptr(x_dev), _ptr(y_dev)))

    def single_layer_dense(self, which, inverse, out_dev, ld=None):
        """Dense float32 single-layer matrix of a surface (or its inverse) into out_dev, a
        device float32 array of shape (n_surface, ld)."""
        n = self.n_m if which == GAMMA_M else self.n_s
        _check(load().pbfb_single_layer_dense(self.h, which, int(inverse), _ptr(out_dev), ld or n))

    def fem_rows(self):
        rp = np.zeros(self.n_v + 1, np.int32)
        col = np.zeros(self.fem_nnz, np.int32)
        val = np.zeros(self.fem_nnz)
        _check(load().pbfb_fem_rows(self.h, _ptr(rp), _ptr(col), _ptr(val)))
        return rp, col, val

    def gmres(self, b_dev, x_dev, tol, restart=200, maxit=1000, precond=JACOBI, inner_iters=30):
        it = ctypes.c_int()
        rel = ctypes.c_double()
        _check(load().pbfb_gmres(self.h, _ptr(b_dev), _ptr(x_dev), tol, restart, maxit, precond,
                                 inner_iters, ctypes.byref(it), ctypes.byref(rel)))
        return it.value, rel.value

    def omega_eval(self, scheme, u_dev, du_dev, c_dev, p_dev, omegas):
        om = np.ascontiguousarray(omegas, np.float64).reshape(-1)
        out = np.zeros((om.size, 8))
        _check(load().pbfb_omega_eval(self.h, scheme, _ptr(u_dev), _ptr(du_dev), _ptr(c_dev),
                                      _ptr(p_dev), _ptr(om), om.size, _ptr(out)))
        return out

    def energy(self, xL_dev, xNL_dev):
        out = np.zeros(4)
        _check(load().pbfb_energy(self.h, _ptr(xL_dev), _ptr(xNL_dev), _ptr(out)))
        return out

    def set_tuning(self, targets_per_thread=0, blocks_per_sm=0, packed=0):
        _check(load().pbfb_set_tuning(self.h, targets_per_thread, blocks_per_sm, packed))

    def get_tuning(self):
        t = Tuning()
        _check(load().pbfb_get_tuning(self.h, ctypes.byref(t)))
        return t.as_dict()

    def apply_tuning(self, d):
        t = Tuning(**{k: int(v) for k, v in d.items()})
        _check(load().pbfb_apply_tuning(self.h, ctypes.byref(t)))

    def autotune(self, reps=3, cache_file=None):
        """Time the candidate launch shapes on this mesh (pbfb_autotune) and apply the fastest.
        With cache_file (JSON), a result stored for the same GPU and size bucket is applied
        instead of timing, and new results are added to the file.  Returns (shapes, ms)."""
        import json
        key = None
        if cache_file is not None:
            import torch
            b = lambda v: int(round(np.log2(max(int(v), 1))))
            key = f"{torch.cuda.get_device_name()}|nm{b(self.n_m)}|ns{b(self.n_s)}|nv{b(self.n_v)}"
            cache = json.load(open(cache_file)) if os.path.exists(cache_file) else {}
            if key in cache:
                self.apply_tuning(cache[key]["shapes"])
                return cache[key]["shapes"], cache[key]["ms"]
        t = Tuning()
        ms = np.zeros(4)
        _check(load().pbfb_autotune(self.h, int(reps), ctypes.byref(t), _ptr(ms)))
        shapes, times = t.as_dict(), dict(nbody_f32=ms[0], nbody_ff=ms[1], spmv=ms[2], inner_pcg=ms[3])
        if key is not None:
            cache = json.load(open(cache_file)) if os.path.exists(cache_file) else {}
            cache[key] = {"shapes": shapes, "ms": times}
            with open(cache_file, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
        return shapes, times

    def profile(self, enable=True, reset=False):
        st = np.zeros(20)
        _check(load().pbfb_profile(self.h, int(enable), int(reset), _ptr(st)))
        return dict(launches=st[0], nbody_launches=st[1], nbody_ms=st[2], nbody_pairs=st[3],
                    spmv_launches=st[4], spmv_ms=st[5], elem_launches=st[6], elem_ms=st[7],
                    nbody_flops=st[8], nbody64_launches=st[9], nbody64_ms=st[10], nbody64_pairs=st[11],
                    nbodyff_launches=st[12], nbodyff_ms=st[13], nbodyff_pairs=st[14],
                    dense_build_ms=st[15], setup_validate_ms=st[16], setup_surfaces_ms=st[17],
                    setup_pattern_ms=st[18], setup_device_ms=st[19])

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().pbfb_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owner of a pbfb_server: queued requests, HBM-budget admission, concurrent solves."""

    def __init__(self, budget_bytes, max_inflight=4, device=0, cached_meshes=0):
        h = ctypes.c_void_p()
        _check(load().pbfb_server_create(device, int(budget_bytes), max_inflight, int(cached_meshes),
                                         ctypes.byref(h)))
        self.h = h

    def submit(self, case, rid, eps_in=None, eps_out=None, kappa=None, T=None, opts=None):
        """Queue a solve of an inputs.Case (arrays are copied by the call)."""
        arrs = [np.ascontiguousarray(case.xyz, np.float64), np.ascontiguousarray(case.tets, np.int32),
                np.ascontiguousarray(case.gm_tris, np.int32), np.ascontiguousarray(case.gs_tris, np.int32),
                np.ascontiguousarray(case.q_xyz, np.float64), np.ascontiguousarray(case.q_z, np.float64)]
        x, t, gm, gs, qx, qz = arrs
        region = getattr(case, "tet_region", None)
        reg = None if region is None else np.ascontiguousarray(region, np.int32)
        r = Request(rid, _ptr(x), x.shape[0], _ptr(t), t.shape[0], _ptr(gm), gm.shape[0], _ptr(gs), gs.shape[0],
                    _ptr(qx), _ptr(qz), qz.shape[0],
                    case.eps_in if eps_in is None else eps_in, case.eps_out if eps_out is None else eps_out,
                    case.kappa if kappa is None else kappa, case.T if T is None else T,
                    ctypes.pointer(opts) if opts is not None else None, None if reg is None else _ptr(reg))
        _check(load().pbfb_server_submit(self.h, ctypes.byref(r)))

    def poll(self, max_n=64, timeout_us=0):
        """Completed responses (at most max_n), waiting up to timeout_us for the first; [] when the
        wait ends empty (PBFB_ERR_TIMEOUT)."""
        buf = (Response * max_n)()
        n = ctypes.c_int()
        code = load().pbfb_server_poll(self.h, buf, max_n, timeout_us, ctypes.byref(n))
        if code == ERR_TIMEOUT:
            return []
        _check(code)
        return [buf[i].as_dict() for i in range(n.value)]

    def stats(self):
        st = np.zeros(8)
        _check(load().pbfb_server_stats(self.h, _ptr(st)))
        return dict(submitted=st[0], completed=st[1], queued=st[2], in_use=st[3], peak=st[4], budget=st[5],
                    mesh_hits=st[6], resident_meshes=st[7])

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().pbfb_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(meshes, params, max_concurrent=4):
    """Solve several meshes (charges set) concurrently; params: list of (eps_in, eps_out, kappa, T, opts)."""
    n = len(meshes)
    hs = (ctypes.c_void_p * n)(*[m.h.value for m in meshes])
    keep = [p[4] for p in params]
    bp = (BatchParams * n)(*[BatchParams(p[0], p[1], p[2], p[3],
                                         ctypes.pointer(p[4]) if p[4] is not None else None) for p in params])
    res = (Result * n)()
    _check(load().pbfb_solve_batch(hs, bp, n, max_concurrent, res))
    del keep
    return [res[i].as_dict() for i in range(n)]
