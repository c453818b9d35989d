"""ctypes binding of libpd_b300.so (declared in include/pd_b300.h).

Argument marshalling only: every function below forwards to the C entry point
of the same name. Arrays may be torch tensors (CUDA or CPU) or numpy arrays;
they must be contiguous float64 (int32 / uint8 for mesh indices / pins). The
library must be built (``paper_2605_14526_b300.build.build()``); a missing
library raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_int32, c_int64, c_uint8, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpd_b300.so")

PD_OK = 0
STATUS = {0: "PD_OK", 1: "PD_ERR_ARG", 2: "PD_ERR_MESH", 3: "PD_ERR_NOT_FACTORED", 4: "PD_ERR_NOT_SPD",
          5: "PD_ERR_NOT_CONVERGED", 6: "PD_ERR_NUMERIC", 7: "PD_ERR_TIMEOUT", 8: "PD_ERR_CUDA",
          9: "PD_ERR_OOM", 10: "PD_ERR_NO_CHECKPOINT", 11: "PD_ERR_TOO_LARGE"}
PD_COROTATED, PD_NEOHOOKEAN, PD_COROT_VOLUME, PD_COROT_LOGVOL = 0, 1, 2, 3
MODELS = {"corotated": PD_COROTATED, "neohookean": PD_NEOHOOKEAN, "corotated_volume": PD_COROT_VOLUME,
          "corotated_logvol": PD_COROT_LOGVOL}
PD_TR_ADAPT, PD_TR_NONE, PD_TR_CLAMP, PD_TR_ABS = 0, 1, 2, 3
PD_SOLVE_AUTO, PD_SOLVE_S, PD_SOLVE_T = 0, 1, 2


class pd_mesh(ctypes.Structure):
    _fields_ = [("n_v", c_int32), ("n_e", c_int32), ("X", c_void_p), ("tets", c_void_p), ("pinned", c_void_p)]


class pd_material(ctypes.Structure):
    _fields_ = [("model", c_int32), ("E", c_void_p), ("nu", c_double), ("density", c_double),
                ("alpha", c_double), ("beta0", c_double), ("gravity", c_double * 3)]


class pd_options(ctypes.Structure):
    _fields_ = [("aa_m", c_int32), ("k_max", c_int32), ("fixed_iters", c_int32), ("local_fp32", c_int32),
                ("tr_mode", c_int32), ("adj_max_iters", c_int32), ("persistent", c_int32),
                ("eps_step", c_double), ("eps_res", c_double),
                ("eps_abs", c_double), ("eps_tr", c_double), ("adj_tol", c_double),
                ("escalate_window", c_int32), ("warm_start", c_int32), ("solve_fp64", c_int32),
                ("wait_polls", c_int32), ("solve_mode", c_int32)]


class pd_stats(ctypes.Structure):
    _fields_ = [("steps", c_int32), ("iters_total", c_int32), ("iters_max", c_int32), ("aa_resets", c_int32),
                ("not_converged", c_int32), ("tau_half", c_int32), ("tau_one", c_int32),
                ("adj_iters_total", c_int32), ("adj_iters_max", c_int32), ("adj_not_converged", c_int32),
                ("status_flags", c_int32), ("n_free", c_int32), ("factor_nnz", c_int64),
                ("factor_seconds", c_double), ("last_rho", c_double), ("launches", c_int64),
                ("escalations", c_int32), ("warm_fallbacks", c_int32),
                ("fwd_device_seconds", c_double), ("bwd_device_seconds", c_double),
                ("contact_iters", c_int32), ("contact_unconverged", c_int32),
                ("solve_mode", c_int32), ("solve_levels", c_int32), ("nnz_L", c_int64)]


class pd_contact_desc(ctypes.Structure):
    _fields_ = [("n_ground", c_int32), ("n_box", c_int32), ("ground", c_void_p), ("box", c_void_p),
                ("ground_z", c_double), ("box_z0", c_double), ("box_travel", c_double), ("box_steps", c_int32),
                ("mu", c_double), ("tol", c_double), ("max_iters", c_int32), ("n_attach", c_int32),
                ("attach", c_void_p), ("attach_target", c_void_p), ("attach_travel", c_void_p),
                ("attach_steps", c_int32)]


class pd_profile_out(ctypes.Structure):
    _fields_ = [("local_launches", c_int64), ("local_ms", c_double), ("solve_launches", c_int64),
                ("solve_ms", c_double), ("phase_ms", c_double * 8), ("work_ms", c_double * 8),
                ("work_max_ms", c_double * 8), ("last_ms", c_double * 8)]


class pd_tuning(ctypes.Structure):
    _fields_ = [("fwd_blocks_per_sm", c_int32), ("bwd_blocks_per_sm", c_int32), ("fwd_grid", c_int32),
                ("bwd_grid", c_int32), ("fwd_gamma", c_double), ("bwd_gamma", c_double),
                ("fwd_min_items", c_int32), ("bwd_min_items", c_int32), ("fwd_ms", c_double), ("bwd_ms", c_double),
                ("candidates", c_int32), ("reserved", c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


class pd_lbfgs_options(ctypes.Structure):
    _fields_ = [("m", c_int32), ("max_iters", c_int32), ("max_evals", c_int32), ("max_ls", c_int32),
                ("gtol", c_double), ("ftol", c_double), ("c1", c_double), ("c2", c_double), ("step0", c_double)]


PD_LBFGS_EVAL, PD_LBFGS_ITERATE, PD_LBFGS_CONVERGED, PD_LBFGS_STOP, PD_LBFGS_FAILED = 1, 2, 3, 4, 5
LBFGS_TASKS = {1: "eval", 2: "iterate", 3: "converged", 4: "stop", 5: "failed"}

_lib = None


def lib():
    """Load the library (once). Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2605_14526_b300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        P = c_void_p
        sig = {
            "pd_default_options": (None, [P]),
            "pd_create": (c_int, [P, P, c_double, P, P]),
            "pd_set_materials": (c_int, [P, P, c_double]),
            "pd_factor": (c_int, [P]),
            "pd_rollout": (c_int, [P, c_int32, P, P, P, c_int64, P, P, P]),
            "pd_step": (c_int, [P, P, P, P, P, P, P]),
            "pd_backward": (c_int, [P, P, P, P, P, P, P, P, c_int64, P]),
            "pd_get_mass": (c_int, [P, P]),
            "pd_get_tau": (c_int, [P, P, c_int32]),
            "pd_get_contact_impulses": (c_int, [P, c_int32, P, P, P, P]),
            "pd_get_checkpoint": (c_int, [P, c_int32, P]),
            "pd_get_stats": (c_int, [P, P]),
            "pd_solve": (c_int, [P, P, P, P]),
            "pd_local_rhs": (c_int, [P, P, P, P]),
            "pd_set_warm_start": (c_int, [P, c_int32]),
            "pd_solve_noalloc": (c_int, [P, P, P, P]),
            "pd_profile": (c_int, [P, c_int32]),
            "pd_get_profile": (c_int, [P, P]),
            "pd_last_error": (ctypes.c_char_p, [P]),
            "pd_destroy": (None, [P]),
            "pd_version": (ctypes.c_char_p, []),
            "pd_reserve": (c_int, [P, c_int32]),
            "pd_rollout_enqueue": (c_int, [P, c_int32, P, P, P, c_int64, P, P, P]),
            "pd_backward_enqueue": (c_int, [P, P, P, P, P, P, P, P, c_int64, P]),
            "pd_collect": (c_int, [P, P]),
            "pd_create_batch": (c_int, [c_int32, P, P, c_double, P, P]),
            "pd_batch_info": (c_int, [P, P, P, P]),
            "pd_set_materials_batch": (c_int, [P, P, P]),
            "pd_get_instance_stats": (c_int, [P, c_int32, P]),
            "pd_batch_teams": (c_int, [P, P, P]),
            "pd_autotune": (c_int, [P, c_int32, P, P, P, c_int64, P, P]),
            "pd_get_tuning": (c_int, [P, P]),
            "pd_set_tuning": (c_int, [P, P]),
            "pd_mlp_create": (c_int, [P, P, P]),
            "pd_mlp_params": (c_int, [P, P, P]),
            "pd_mlp_fit_normalization": (c_int, [P, P, P, c_int64, P]),
            "pd_mlp_forward": (c_int, [P, P, P, c_int64, P]),
            "pd_mlp_grad": (c_int, [P, P, P, c_int64, P, P, P]),
            "pd_mlp_train_step": (c_int, [P, P, P, c_int64, c_double, P, P]),
            "pd_mlp_last_error": (ctypes.c_char_p, [P]),
            "pd_mlp_destroy": (None, [P]),
            "pd_mlp_sample": (c_int, [P, P, P, P, P, P, P]),
            "pd_mlp_load": (c_int, [P, P, ctypes.c_size_t]),
            "pd_warm_start": (c_int, [P, P, P, P, P]),
            "pd_set_contacts": (c_int, [P, P]),
            "pd_lbfgs_default_options": (None, [P]),
            "pd_lbfgs_create": (c_int, [c_int32, P, P]),
            "pd_lbfgs_next": (c_int, [P, P, c_double, P, P]),
            "pd_lbfgs_info": (c_int, [P, P, P, P, P]),
            "pd_lbfgs_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class PDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _ptr(a, dtype=np.float64):
    """Address of a contiguous array (torch tensor or numpy), or None."""
    if a is None:
        return None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            want = {np.float64: torch.float64, np.float32: torch.float32, np.int32: torch.int32,
                    np.uint8: torch.uint8}[dtype]
            if a.dtype != want or not a.is_contiguous():
                raise TypeError(f"tensor must be contiguous {want}")
            return a.data_ptr()
    except ImportError:
        pass
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"array must be a C-contiguous {np.dtype(dtype).name} ndarray")
    return a.ctypes.data


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(ctx, code):
    if code != PD_OK:
        msg = lib().pd_last_error(ctx).decode() if ctx else ""
        raise PDError(code, msg)


# ---------------------------------------------------------------- same names

def pd_default_options() -> pd_options:
    o = pd_options()
    lib().pd_default_options(ctypes.byref(o))
    return o


def pd_create(X, tets, pinned, E, model, nu, density, alpha, beta0, gravity, dt, options: pd_options):
    """Returns an opaque context handle; the host arrays are copied by the library."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    E = np.ascontiguousarray(E, dtype=np.float64)
    pin = None if pinned is None else np.ascontiguousarray(pinned, dtype=np.uint8)
    mesh = pd_mesh(int(X.shape[0]), int(tets.shape[0]), _ptr(X), _ptr(tets, np.int32),
                   None if pin is None else _ptr(pin, np.uint8))
    mat = pd_material(int(model), _ptr(E), float(nu), float(density), float(alpha), float(beta0),
                      (c_double * 3)(*[float(g) for g in gravity]))
    out = c_void_p()
    code = lib().pd_create(ctypes.byref(mesh), ctypes.byref(mat), float(dt), ctypes.byref(options), ctypes.byref(out))
    if code != PD_OK:
        msg = lib().pd_last_error(out).decode() if out.value else ""
        if out.value:
            lib().pd_destroy(out)
        raise PDError(code, msg)
    return out


def pd_set_materials(ctx, E, nu):
    E = np.ascontiguousarray(E, dtype=np.float64)
    _check(ctx, lib().pd_set_materials(ctx, _ptr(E), float(nu)))


def pd_factor(ctx):
    _check(ctx, lib().pd_factor(ctx))


def pd_rollout(ctx, T, q0, v0, f_ext, f_stride, qT, vT, stream=None, check=True):
    code = lib().pd_rollout(ctx, int(T), _ptr(q0), _ptr(v0), _ptr(f_ext), int(f_stride), _ptr(qT), _ptr(vT),
                            _stream(stream))
    if check:
        _check(ctx, code)
    return code


def pd_step(ctx, q_t, v_t, f_ext, q_next, v_next, stream=None):
    _check(ctx, lib().pd_step(ctx, _ptr(q_t), _ptr(v_t), _ptr(f_ext), _ptr(q_next), _ptr(v_next), _stream(stream)))


def pd_backward(ctx, dqT, dvT, dq0, dv0, dE, dnu, df_ext, df_stride, stream=None, check=True):
    code = lib().pd_backward(ctx, _ptr(dqT), _ptr(dvT), _ptr(dq0), _ptr(dv0), _ptr(dE), _ptr(dnu), _ptr(df_ext),
                             int(df_stride), _stream(stream))
    if check:
        _check(ctx, code)
    return code


def pd_solve(ctx, b, x, stream=None):
    _check(ctx, lib().pd_solve(ctx, _ptr(b), _ptr(x), _stream(stream)))


def pd_local_rhs(ctx, q, out, stream=None):
    _check(ctx, lib().pd_local_rhs(ctx, _ptr(q), _ptr(out), _stream(stream)))


def pd_solve_noalloc(ctx, b, x, stream=None):
    _check(ctx, lib().pd_solve_noalloc(ctx, _ptr(b), _ptr(x), _stream(stream)))


def pd_get_mass(ctx, n_v):
    m = np.zeros(n_v)
    _check(ctx, lib().pd_get_mass(ctx, _ptr(m)))
    return m


def pd_get_checkpoint(ctx, t, n_v):
    q = np.zeros((n_v, 3))
    _check(ctx, lib().pd_get_checkpoint(ctx, int(t), _ptr(q)))
    return q


def pd_get_contact_impulses(ctx, t):
    """(vertex [K], lam_n [K], lam_f [K,2]) of step t of the last rollout."""
    n = ctypes.c_int32(0)
    _check(ctx, lib().pd_get_contact_impulses(ctx, int(t), ctypes.byref(n), None, None, None))
    K = n.value
    v = np.zeros(K, dtype=np.int32)
    ln = np.zeros(K)
    lf = np.zeros((K, 2))
    if K:
        _check(ctx, lib().pd_get_contact_impulses(ctx, int(t), ctypes.byref(n), _ptr(v, np.int32), _ptr(ln), _ptr(lf)))
    return v, ln, lf


def pd_get_tau(ctx, T):
    t = np.zeros(T)
    _check(ctx, lib().pd_get_tau(ctx, _ptr(t), int(T)))
    return t


def pd_get_stats(ctx) -> pd_stats:
    s = pd_stats()
    _check(ctx, lib().pd_get_stats(ctx, ctypes.byref(s)))
    return s


def pd_profile(ctx, enable: bool):
    _check(ctx, lib().pd_profile(ctx, 1 if enable else 0))


def pd_get_profile(ctx) -> pd_profile_out:
    p = pd_profile_out()
    _check(ctx, lib().pd_get_profile(ctx, ctypes.byref(p)))
    return p


def pd_reserve(ctx, T):
    _check(ctx, lib().pd_reserve(ctx, int(T)))


def pd_rollout_enqueue(ctx, T, q0, v0, f_ext, f_stride, qT, vT, stream=None):
    _check(ctx, lib().pd_rollout_enqueue(ctx, int(T), _ptr(q0), _ptr(v0), _ptr(f_ext), int(f_stride), _ptr(qT),
                                         _ptr(vT), _stream(stream)))


def pd_backward_enqueue(ctx, dqT, dvT, dq0, dv0, dE, dnu, df_ext, df_stride, stream=None):
    _check(ctx, lib().pd_backward_enqueue(ctx, _ptr(dqT), _ptr(dvT), _ptr(dq0), _ptr(dv0), _ptr(dE), _ptr(dnu),
                                          _ptr(df_ext), int(df_stride), _stream(stream)))


def pd_collect(ctx, stream=None, check=True):
    code = lib().pd_collect(ctx, _stream(stream))
    if check:
        _check(ctx, code)
    return code


def _mesh_material(scene):
    """pd_mesh / pd_material of a workload, with the arrays they point at."""
    X = np.ascontiguousarray(scene.X, dtype=np.float64)
    tets = np.ascontiguousarray(scene.tets, dtype=np.int32)
    E = np.ascontiguousarray(scene.E, dtype=np.float64)
    pin = np.ascontiguousarray(scene.pinned, dtype=np.uint8)
    model = MODELS[scene.model]
    mesh = pd_mesh(int(X.shape[0]), int(tets.shape[0]), _ptr(X), _ptr(tets, np.int32), _ptr(pin, np.uint8))
    mat = pd_material(model, _ptr(E), float(scene.nu), float(scene.density), float(scene.alpha), float(scene.beta0),
                      (c_double * 3)(*[float(g) for g in scene.gravity]))
    return mesh, mat, (X, tets, E, pin)


def pd_create_batch(scenes, dt, options: pd_options):
    """One context for a list of workloads (each a ``Scene``); arrays are copied."""
    n = len(scenes)
    meshes = (pd_mesh * n)()
    mats = (pd_material * n)()
    keep = []
    for i, sc in enumerate(scenes):
        m, t, arrays = _mesh_material(sc)
        meshes[i] = m
        mats[i] = t
        keep.append(arrays)
    out = c_void_p()
    code = lib().pd_create_batch(n, meshes, mats, float(dt), ctypes.byref(options), ctypes.byref(out))
    if code != PD_OK:
        msg = lib().pd_last_error(out).decode() if out.value else ""
        if out.value:
            lib().pd_destroy(out)
        raise PDError(code, msg)
    return out


def pd_batch_info(ctx):
    n = c_int32()
    _check(ctx, lib().pd_batch_info(ctx, ctypes.byref(n), None, None))
    v_off = np.zeros(n.value + 1, dtype=np.int64)
    e_off = np.zeros(n.value + 1, dtype=np.int64)
    _check(ctx, lib().pd_batch_info(ctx, ctypes.byref(n), v_off.ctypes.data, e_off.ctypes.data))
    return n.value, v_off, e_off


def pd_set_materials_batch(ctx, E, nu):
    E = np.ascontiguousarray(E, dtype=np.float64)
    nu = np.ascontiguousarray(nu, dtype=np.float64)
    _check(ctx, lib().pd_set_materials_batch(ctx, _ptr(E), _ptr(nu)))


def pd_get_instance_stats(ctx, i) -> pd_stats:
    s = pd_stats()
    _check(ctx, lib().pd_get_instance_stats(ctx, int(i), ctypes.byref(s)))
    return s


def pd_batch_teams(ctx, n):
    f = np.zeros(n, dtype=np.int32)
    b = np.zeros(n, dtype=np.int32)
    _check(ctx, lib().pd_batch_teams(ctx, f.ctypes.data, b.ctypes.data))
    return f, b


def pd_autotune(ctx, T_probe, q0, v0, f_ext, f_stride, stream=None) -> pd_tuning:
    t = pd_tuning()
    _check(ctx, lib().pd_autotune(ctx, int(T_probe), _ptr(q0), _ptr(v0), _ptr(f_ext), int(f_stride),
                                  ctypes.byref(t), _stream(stream)))
    return t


def pd_get_tuning(ctx) -> pd_tuning:
    t = pd_tuning()
    _check(ctx, lib().pd_get_tuning(ctx, ctypes.byref(t)))
    return t


def pd_set_tuning(ctx, t: pd_tuning):
    _check(ctx, lib().pd_set_tuning(ctx, ctypes.byref(t)))


MLP_PARAMS, MLP_NORM = 34435, 17


def _mcheck(net, code):
    if code != PD_OK:
        msg = lib().pd_mlp_last_error(net).decode() if net else ""
        raise PDError(code, msg)


def pd_mlp_create(theta, norm):
    theta = np.ascontiguousarray(theta, dtype=np.float32)
    norm = np.ascontiguousarray(norm, dtype=np.float32)
    if theta.size != MLP_PARAMS or norm.size != MLP_NORM:
        raise ValueError("theta must hold 34435 and norm 17 values")
    out = c_void_p()
    code = lib().pd_mlp_create(_ptr(theta, np.float32), _ptr(norm, np.float32), ctypes.byref(out))
    if code != PD_OK:
        msg = lib().pd_mlp_last_error(out).decode() if out.value else ""
        if out.value:
            lib().pd_mlp_destroy(out)
        raise PDError(code, msg)
    return out


def pd_mlp_params(net):
    theta = np.zeros(MLP_PARAMS, dtype=np.float32)
    norm = np.zeros(MLP_NORM, dtype=np.float32)
    _mcheck(net, lib().pd_mlp_params(net, _ptr(theta, np.float32), _ptr(norm, np.float32)))
    return theta, norm


def pd_mlp_fit_normalization(net, feat, targ, n, stream=None):
    _mcheck(net, lib().pd_mlp_fit_normalization(net, _ptr(feat, np.float32), _ptr(targ, np.float32), int(n),
                                                _stream(stream)))


def pd_mlp_forward(net, feat, r, n, stream=None):
    _mcheck(net, lib().pd_mlp_forward(net, _ptr(feat, np.float32), _ptr(r, np.float32), int(n), _stream(stream)))


def pd_mlp_grad(net, feat, targ, n, grad=None, stream=None) -> float:
    loss = c_double()
    _mcheck(net, lib().pd_mlp_grad(net, _ptr(feat, np.float32), _ptr(targ, np.float32), int(n),
                                   _ptr(grad, np.float32), ctypes.byref(loss), _stream(stream)))
    return loss.value


def pd_mlp_train_step(net, feat, targ, n, lr, stream=None, want_loss=True):
    loss = c_double()
    _mcheck(net, lib().pd_mlp_train_step(net, _ptr(feat, np.float32), _ptr(targ, np.float32), int(n), float(lr),
                                         ctypes.byref(loss) if want_loss else None, _stream(stream)))
    return loss.value if want_loss else None


def pd_mlp_destroy(net):
    if net is not None and net.value:
        lib().pd_mlp_destroy(net)


def pd_mlp_sample(ctx, x_tm1, x_t, x_tp1, feat, targ, stream=None):
    _check(ctx, lib().pd_mlp_sample(ctx, _ptr(x_tm1), _ptr(x_t), _ptr(x_tp1), _ptr(feat, np.float32),
                                    _ptr(targ, np.float32), _stream(stream)))


def pd_lbfgs_default_options() -> pd_lbfgs_options:
    o = pd_lbfgs_options()
    lib().pd_lbfgs_default_options(ctypes.byref(o))
    return o


def pd_lbfgs_create(n, options: pd_lbfgs_options | None = None):
    out = c_void_p()
    code = lib().pd_lbfgs_create(int(n), ctypes.byref(options) if options is not None else None, ctypes.byref(out))
    if code != PD_OK:
        raise PDError(code, "pd_lbfgs_create")
    return out


def pd_lbfgs_next(opt, x, f, g):
    """x: float64 ndarray [n] (updated in place); g may be None right after
    an ITERATE task. Returns the task code."""
    task = c_int32()
    code = lib().pd_lbfgs_next(opt, _ptr(x), float(f), _ptr(g), ctypes.byref(task))
    if code != PD_OK:
        raise PDError(code, "pd_lbfgs_next")
    return task.value


def pd_lbfgs_info(opt):
    it, ev, f, gm = c_int32(), c_int32(), c_double(), c_double()
    _check(None, lib().pd_lbfgs_info(opt, ctypes.byref(it), ctypes.byref(ev), ctypes.byref(f), ctypes.byref(gm)))
    return {"iters": it.value, "evals": ev.value, "f": f.value, "gmax": gm.value}


def pd_lbfgs_destroy(opt):
    if opt is not None and opt.value:
        lib().pd_lbfgs_destroy(opt)


def pd_mlp_load(ctx, blob):
    blob = np.ascontiguousarray(blob, dtype=np.float32)
    _check(ctx, lib().pd_mlp_load(ctx, _ptr(blob, np.float32), blob.nbytes))


def pd_set_warm_start(ctx, mode):
    _check(ctx, lib().pd_set_warm_start(ctx, int(mode)))


def pd_warm_start(ctx, x_t, x_tm1, q0, stream=None):
    _check(ctx, lib().pd_warm_start(ctx, _ptr(x_t), _ptr(x_tm1), _ptr(q0), _stream(stream)))


def contact_desc(spec, tol=0.0, max_iters=0):
    """(pd_contact_desc, arrays) for an ``inputs.ContactSpec``: the
    descriptor points into the returned arrays, which must outlive its use."""
    g = np.ascontiguousarray(spec.ground, dtype=np.int32)
    b = np.ascontiguousarray(spec.box, dtype=np.int32)
    a = np.ascontiguousarray(spec.attach, dtype=np.int32)
    p0 = np.ascontiguousarray(spec.attach_p0, dtype=np.float64).reshape(-1, 3)
    tr = np.ascontiguousarray(spec.attach_travel, dtype=np.float64).reshape(-1, 3)
    if p0.shape[0] != a.size or tr.shape[0] != a.size:
        raise ValueError("attach_p0 and attach_travel need one row per attached vertex")
    desc = pd_contact_desc(int(g.size), int(b.size), _ptr(g, np.int32) if g.size else None,
                           _ptr(b, np.int32) if b.size else None, float(spec.ground_z), float(spec.box_z0),
                           float(spec.box_travel), int(spec.box_steps), float(spec.mu), float(tol), int(max_iters),
                           int(a.size), _ptr(a, np.int32) if a.size else None, _ptr(p0) if a.size else None,
                           _ptr(tr) if a.size else None, int(spec.attach_steps))
    return desc, (g, b, a, p0, tr)


def pd_set_contacts(ctx, spec, tol=0.0, max_iters=0):
    """Contacts of a workload (``inputs.ContactSpec``), or None to remove them."""
    if spec is None:
        _check(ctx, lib().pd_set_contacts(ctx, None))
        return
    desc, arrays = contact_desc(spec, tol, max_iters)   # arrays: the data desc points into, alive through the call
    _check(ctx, lib().pd_set_contacts(ctx, ctypes.byref(desc)))


def pd_last_error(ctx) -> str:
    return lib().pd_last_error(ctx).decode()


def pd_destroy(ctx):
    if ctx is not None and ctx.value:
        lib().pd_destroy(ctx)


def pd_version() -> str:
    return lib().pd_version().decode()


# ------------------------------------------------------------ convenience

def options_for(settings) -> pd_options:
    """pd_options from a workload's SolverSettings."""
    o = pd_default_options()
    o.aa_m = settings.aa_m
    o.k_max = settings.k_max
    o.fixed_iters = settings.fixed_iters
    o.local_fp32 = 1 if settings.local_fp32 else 0
    o.tr_mode = settings.tr_mode
    o.eps_step = settings.eps_step
    o.eps_res = settings.eps_res
    o.eps_abs = settings.eps_abs
    o.eps_tr = settings.eps_tr
    o.solve_fp64 = 1 if getattr(settings, "solve_fp64", False) else 0
    o.solve_mode = int(getattr(settings, "solve_mode", PD_SOLVE_AUTO))
    return o


class PDContext:
    """Owns one pd_ctx for a workload (``paper_2605_14526_b300.inputs.Scene``)."""

    def __init__(self, scene, options: pd_options | None = None, factor: bool = True):
        self.scene = scene
        self.options = options or options_for(scene.solver)
        model = MODELS[scene.model]
        self.ctx = pd_create(scene.X, scene.tets, scene.pinned, scene.E, model, scene.nu, scene.density,
                             scene.alpha, scene.beta0, scene.gravity, scene.dt, self.options)
        self.n_v, self.n_e = scene.n_v, scene.n_e
        if getattr(scene, "contact", None) is not None:
            pd_set_contacts(self.ctx, scene.contact)
        if factor:
            pd_factor(self.ctx)

    def close(self):
        pd_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            if getattr(self, "ctx", None) is not None:
                self.close()
        except Exception:
            pass

    def set_materials(self, E, nu):
        pd_set_materials(self.ctx, E, nu)
        pd_factor(self.ctx)

    def ensure_materials(self, E, nu):
        """Set (and refactor) only if E [n_e] or nu [1] differ from the current ones."""
        nu_f = float(np.asarray(nu).reshape(-1)[0])
        if not (np.array_equal(E, self.scene.E) and nu_f == self.scene.nu):
            self.set_materials(E, nu_f)
            self.scene = self.scene.replace(E=np.array(E, dtype=np.float64), nu=nu_f)

    def stats(self):
        return pd_get_stats(self.ctx)

    def mass(self):
        return pd_get_mass(self.ctx, self.n_v)


class BatchContext:
    """Owns one batched pd_ctx for a list of workloads (all with one dt and one
    set of options); arrays at the boundary are the concatenation over
    instances (``v_off`` / ``e_off`` prefix offsets)."""

    def __init__(self, scenes, options: pd_options | None = None, factor: bool = True):
        self.scenes = list(scenes)
        self.options = options or options_for(self.scenes[0].solver)
        self.ctx = pd_create_batch(self.scenes, self.scenes[0].dt, self.options)
        self.n, self.v_off, self.e_off = pd_batch_info(self.ctx)
        self.n_v, self.n_e = int(self.v_off[-1]), int(self.e_off[-1])
        self.E = self.concat([sc.E for sc in self.scenes])
        self.nu = np.array([sc.nu for sc in self.scenes], dtype=np.float64)
        if factor:
            pd_factor(self.ctx)

    def close(self):
        pd_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            if getattr(self, "ctx", None) is not None:
                self.close()
        except Exception:
            pass

    def concat(self, arrays):
        return np.concatenate([np.asarray(a, dtype=np.float64).reshape(-1) for a in arrays])

    def split_v(self, a):
        a = np.asarray(a).reshape(self.n_v, -1)
        return [a[self.v_off[i]:self.v_off[i + 1]] for i in range(self.n)]

    def split_e(self, a):
        a = np.asarray(a).reshape(-1)
        return [a[self.e_off[i]:self.e_off[i + 1]] for i in range(self.n)]

    def set_materials(self, E, nu):
        pd_set_materials_batch(self.ctx, E, nu)
        pd_factor(self.ctx)
        self.E = np.array(E, dtype=np.float64).reshape(-1)
        self.nu = np.array(nu, dtype=np.float64).reshape(-1)

    def ensure_materials(self, E, nu):
        """Set (and refactor) only if E [sum n_e] or nu [n] differ from the current ones."""
        nu = np.asarray(nu, dtype=np.float64).reshape(-1)
        if not (np.array_equal(E, self.E) and np.array_equal(nu, self.nu)):
            self.set_materials(E, nu)

    def teams(self):
        """Blocks per instance of the forward and adjoint launches."""
        return pd_batch_teams(self.ctx, self.n)

    def stats(self):
        return pd_get_stats(self.ctx)

    def instance_stats(self, i):
        return pd_get_instance_stats(self.ctx, i)

    def mass(self):
        return pd_get_mass(self.ctx, self.n_v)


class MLP:
    """Owns one pd_mlp trainer (warm-start network) on the current device."""

    def __init__(self, theta, norm):
        self.net = pd_mlp_create(theta, norm)

    def close(self):
        pd_mlp_destroy(self.net)
        self.net = None

    def __del__(self):
        try:
            if getattr(self, "net", None) is not None:
                self.close()
        except Exception:
            pass

    def params(self):
        return pd_mlp_params(self.net)

    def blob(self):
        """FP32 parameters followed by the normalisation, as pd_mlp_load takes them."""
        theta, norm = self.params()
        return np.concatenate([theta, norm]).astype(np.float32)
