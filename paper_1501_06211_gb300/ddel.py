"""ctypes binding of libddel (include/ddel.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module only
converts Python/NumPy/torch arguments into the plain pointers and structs of
the C ABI.  The functions keep the C names (``ddel_create``, ``ddel_solve``,
...); ``Solver`` is a thin convenience wrapper over them.  Importing this
module fails loudly when libddel.so has not been built.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libddel.so")

c_int, c_double, c_void_p, c_uint32, c_int64 = (ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                                  ctypes.c_uint32, ctypes.c_int64)

DDEL_OK, DDEL_EINVAL, DDEL_ENOMEM, DDEL_ECUDA = 0, -1, -2, -3
DDEL_ENOTSPD, DDEL_ENOCONV, DDEL_EBREAKDOWN, DDEL_ESTATE, DDEL_ETIMEOUT = -4, -5, -6, -7, -8
DDEL_FP64, DDEL_FP32, DDEL_MIXED = 0, 1, 2
DDEL_X0_ZERO, DDEL_X0_WARM = 0, 1
DDEL_COARSE_X0, DDEL_COARSE_CORRECT, DDEL_COARSE_DEFLATE = 1, 2, 4
DDEL_MAX_COARSE = 8


class ddel_mesh(ctypes.Structure):
    _fields_ = [("dim", c_int), ("nx", c_int), ("ny", c_int), ("nz", c_int), ("sub", c_int)]


class ddel_material(ctypes.Structure):
    _fields_ = [("E", c_double), ("nu", c_double), ("plane_stress", c_int), ("simp_p", c_double),
                ("rho_min", c_double)]


class ddel_bc(ctypes.Structure):
    _fields_ = [("clamp_faces", c_uint32), ("fixed_dof", c_void_p), ("n_point", c_int),
                ("point_node", c_void_p), ("point_force", c_void_p), ("traction_face", c_int),
                ("traction", c_double * 3), ("body_force", c_double * 3)]


class ddel_options(ctypes.Structure):
    _fields_ = [("precision", c_int), ("theta", c_double), ("face_scaling", c_int),
                ("crosspoint_mode", c_int), ("tol", c_double), ("max_it", c_int),
                ("max_cycles", c_int), ("inner_tol", c_double), ("x0_mode", c_int),
                ("schur_mode", c_int), ("use_graph", c_int), ("check_every", c_int),
                ("tensor_form", c_int),
                ("schur_split", c_int), ("relax_switch", c_double), ("relax_delta", c_double)]


def _set_fields(opt, options):
    """Copies keyword options into an options structure; a name that is not
    one of its fields raises (ctypes would keep it as a plain attribute that
    the library never sees)."""
    unknown = sorted(set(options) - {k for k, _ in type(opt)._fields_})
    if unknown:
        raise TypeError(f"unknown {type(opt).__name__} field(s): " + ", ".join(unknown))
    for k, v in options.items():
        setattr(opt, k, v)


class ddel_stats(ctypes.Structure):
    _fields_ = [("status", c_int), ("iters", c_int), ("cycles", c_int), ("relres", c_double),
                ("pcg_relres", c_double), ("bad_subdomain", c_int), ("fallback", c_int),
                ("t_factor_ms", c_double),
                ("t_condense_ms", c_double), ("t_pcg_ms", c_double), ("t_backsub_ms", c_double),
                ("t_verify_ms", c_double), ("t_total_ms", c_double), ("coarse_k", c_int),
                ("x0_used", c_int), ("low_iters", c_int), ("replacements", c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ddel_gmres_options(ctypes.Structure):
    _fields_ = [("precond", c_int), ("lanczos_steps", c_int), ("inner_tol", c_double),
                ("mass_tol", c_double), ("global_scaling", c_int), ("tol", c_double), ("max_it", c_int)]


class ddel_gmres_stats(ctypes.Structure):
    _fields_ = [("status", c_int), ("iters", c_int), ("est_relres", c_double), ("relres", c_double),
                ("inner_min", c_int), ("inner_max", c_int), ("inner_mean", c_double),
                ("lanczos_m", c_int), ("t_ms", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


DDEL_PREC_IDENTITY, DDEL_PREC_FACE, DDEL_PREC_GLOBAL = 0, 1, 2
DDEL_MAX_LANCZOS = 32


class ddel_info_t(ctypes.Structure):
    _fields_ = [("dim", c_int), ("n_sub", c_int), ("n_elem", c_int), ("max_block", c_int),
                ("max_blocks_per_sub", c_int), ("n_nodes", c_int64), ("n_dof", c_int64),
                ("n_gamma", c_int64), ("n_fixed", c_int64), ("factor_bytes", c_int64),
                ("n_face_blocks", c_int), ("n_cross", c_int)]


class ddel_kernel_info_t(ctypes.Structure):
    _fields_ = [("launches_total", c_int64), ("launches_since_assemble", c_int64),
                ("schur_apply_bytes", c_int64), ("schur_apply_flops", c_int64),
                ("schur_form", c_int), ("precision", c_int), ("double_float", c_int)]


class ddel_topopt_state(ctypes.Structure):
    _fields_ = [("rho", c_void_p), ("volfrac", c_double), ("r_min", c_double), ("move", c_double),
                ("iteration", c_int), ("compliance", c_double), ("volume", c_double),
                ("change", c_double), ("lambda_", c_double), ("u", c_void_p), ("rho_phys", c_void_p),
                ("learner", c_void_p), ("tol_eta", c_double), ("tol_max", c_double),
                ("tol_used", c_double), ("compliance_prev", c_double)]


class ddel_learner_options(ctypes.Structure):
    _fields_ = [("mode", c_int), ("coarse_flags", c_int), ("k_history", c_int), ("replay", c_int),
                ("train_steps", c_int), ("batch", c_int), ("min_samples", c_int), ("lr", c_double),
                ("widths", c_int * 4), ("seed", ctypes.c_uint64)]


class ddel_learner_info(ctypes.Structure):
    _fields_ = [("samples", c_int), ("predictions", c_int), ("adam_steps", c_int64),
                ("last_loss", c_double), ("t_train_ms", c_double), ("t_predict_ms", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
            " (the solver has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    sig = {
        "ddel_default_options": (None, [P(ddel_options)]),
        "ddel_strerror": (ctypes.c_char_p, [c_int]),
        "ddel_last_error": (ctypes.c_char_p, [c_void_p]),
        "ddel_create": (c_int, [P(ddel_mesh), P(ddel_material), P(ddel_bc), P(ddel_options),
                                c_void_p, P(c_void_p)]),
        "ddel_destroy": (None, [c_void_p]),
        "ddel_get_info": (c_int, [c_void_p, P(ddel_info_t)]),
        "ddel_set_options": (c_int, [c_void_p, P(ddel_options)]),
        "ddel_assemble": (c_int, [c_void_p, c_void_p, c_int]),
        "ddel_factor": (c_int, [c_void_p]),
        "ddel_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_int, P(ddel_stats)]),
        "ddel_apply_K": (c_int, [c_void_p, c_void_p, c_void_p]),
        "ddel_condense": (c_int, [c_void_p, c_void_p, c_void_p]),
        "ddel_schur_apply": (c_int, [c_void_p, c_void_p, c_void_p]),
        "ddel_schur_apply_ring": (c_int, [c_void_p, c_void_p]),
        "ddel_precond_apply": (c_int, [c_void_p, c_void_p, c_void_p]),
        "ddel_back_substitute": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
        "ddel_pcg": (c_int, [c_void_p, c_void_p, c_void_p, c_double, P(ddel_stats)]),
        "ddel_residual_norm": (c_int, [c_void_p, c_void_p, c_void_p, P(c_double), P(c_double)]),
        "ddel_gamma_dofs": (c_int, [c_void_p, c_void_p]),
        "ddel_load_vector": (c_int, [c_void_p, c_void_p]),
        "ddel_fixed_mask": (c_int, [c_void_p, c_void_p]),
        "ddel_kernel_info": (c_int, [c_void_p, P(ddel_kernel_info_t)]),
        "ddel_batch_solve": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
        "ddel_batch_solve_persistent": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
        "ddel_autotune": (c_int, [c_void_p, ctypes.c_char_p, c_void_p, c_void_p, c_void_p]),
        "ddel_topopt_step": (c_int, [c_void_p, P(ddel_topopt_state), P(ddel_stats)]),
        "ddel_set_coarse": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int]),
        "ddel_selftest_wait_timeout": (c_int, [ctypes.c_uint, P(c_int)]),
        "ddel_default_gmres_options": (None, [P(ddel_gmres_options)]),
        "ddel_gmres_solve": (c_int, [c_void_p, P(ddel_gmres_options), c_void_p, c_void_p, c_int,
                                     P(ddel_gmres_stats)]),
        "ddel_global_precond_apply": (c_int, [c_void_p, P(ddel_gmres_options), c_void_p, c_void_p, c_void_p]),
        "ddel_checkpoint_save": (c_int, [c_void_p, P(ddel_topopt_state), ctypes.c_char_p]),
        "ddel_checkpoint_load": (c_int, [c_void_p, P(ddel_topopt_state), ctypes.c_char_p]),
        "ddel_residual_norm_noalloc": (c_int, [c_int, c_int, c_int, c_int, c_void_p, c_void_p,
                                               c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                               c_void_p]),
        "ddel_cnn_create": (c_int, [c_int, c_int, c_int, c_int, c_int, c_void_p, ctypes.c_uint64,
                                    c_void_p, P(c_void_p)]),
        "ddel_cnn_destroy": (None, [c_void_p]),
        "ddel_cnn_last_error": (ctypes.c_char_p, [c_void_p]),
        "ddel_cnn_num_params": (c_int64, [c_void_p]),
        "ddel_cnn_get_params": (c_int, [c_void_p, c_void_p, c_int]),
        "ddel_cnn_set_params": (c_int, [c_void_p, c_void_p, c_int]),
        "ddel_cnn_forward": (c_int, [c_void_p, c_void_p, c_int, c_void_p]),
        "ddel_cnn_loss_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_int, P(c_double), c_void_p]),
        "ddel_cnn_adam_step": (c_int, [c_void_p, c_double, c_double, c_double, c_double]),
        "ddel_learner_default_options": (None, [P(ddel_learner_options)]),
        "ddel_learner_create": (c_int, [c_void_p, P(ddel_learner_options), P(c_void_p)]),
        "ddel_learner_destroy": (None, [c_void_p]),
        "ddel_learner_predict": (c_int, [c_void_p, c_void_p]),
        "ddel_learner_observe": (c_int, [c_void_p, c_void_p, c_void_p]),
        "ddel_learner_get_info": (c_int, [c_void_p, P(ddel_learner_info)]),
        "ddel_learner_features": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
        "ddel_learner_grid": (c_int, [c_void_p, P(c_int), P(c_int)]),
        "ddel_learner_network": (c_void_p, [c_void_p]),
        "ddel_plan_create": (c_int, [P(ddel_mesh), P(ddel_material), P(ddel_bc), c_double,
                                     P(c_void_p)]),
        "ddel_plan_destroy": (None, [c_void_p]),
        "ddel_plan_info": (c_int, [c_void_p, P(ddel_info_t)]),
        "ddel_plan_gamma_dofs": (c_int, [c_void_p, c_void_p]),
        "ddel_plan_face_block": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
        "ddel_plan_interface_operator": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                                 c_void_p, c_void_p, c_void_p]),
        "ddel_plan_element_matrix": (c_int, [c_void_p, c_void_p]),
        "ddel_plan_subdomain": (c_int, [c_void_p, c_int, c_void_p, c_void_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib, sig


_lib, SIGNATURES = _load()
EXPORTED = sorted(SIGNATURES)


class DDELError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__(f"{_lib.ddel_strerror(code).decode()} ({code}) {msg}".strip())


def _check(code, ctx=None):
    if code != DDEL_OK:
        raise DDELError(code, _lib.ddel_last_error(ctx).decode())


def _ptr(a):
    """Device/host pointer of a torch tensor or NumPy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    raise TypeError(type(a))


# ----------------------------------------------------------------- raw C names
def ddel_default_options():
    o = ddel_options()
    _lib.ddel_default_options(ctypes.byref(o))
    return o


def ddel_strerror(code):
    return _lib.ddel_strerror(code).decode()


def ddel_create(mesh, mat, bc, opt, stream=None):
    h = c_void_p()
    code = _lib.ddel_create(ctypes.byref(mesh), ctypes.byref(mat), ctypes.byref(bc),
                            ctypes.byref(opt) if opt is not None else None, stream, ctypes.byref(h))
    return code, h


ddel_destroy = _lib.ddel_destroy


def ddel_get_info(h):
    info = ddel_info_t()
    _check(_lib.ddel_get_info(h, ctypes.byref(info)), h)
    return info


def ddel_set_options(h, opt):
    return _lib.ddel_set_options(h, ctypes.byref(opt))


def ddel_assemble(h, rho, on_device):
    return _lib.ddel_assemble(h, _ptr(rho), int(on_device))


def ddel_factor(h):
    return _lib.ddel_factor(h)


def ddel_solve(h, f, u, on_device):
    st = ddel_stats()
    code = _lib.ddel_solve(h, _ptr(f), _ptr(u), int(on_device), ctypes.byref(st))
    return code, st


def ddel_apply_K(h, x, y):
    return _lib.ddel_apply_K(h, _ptr(x), _ptr(y))


def ddel_condense(h, f, g):
    return _lib.ddel_condense(h, _ptr(f), _ptr(g))


def ddel_schur_apply(h, x, y):
    return _lib.ddel_schur_apply(h, _ptr(x), _ptr(y))


def ddel_schur_apply_ring(h, x):
    return _lib.ddel_schur_apply_ring(h, _ptr(x))


def ddel_precond_apply(h, r, z):
    return _lib.ddel_precond_apply(h, _ptr(r), _ptr(z))


def ddel_back_substitute(h, f, uG, u):
    return _lib.ddel_back_substitute(h, _ptr(f), _ptr(uG), _ptr(u))


def ddel_pcg(h, g, x, tol_abs):
    st = ddel_stats()
    code = _lib.ddel_pcg(h, _ptr(g), _ptr(x), float(tol_abs), ctypes.byref(st))
    return code, st


def ddel_residual_norm(h, f, u):
    rn, fn = c_double(), c_double()
    code = _lib.ddel_residual_norm(h, _ptr(f), _ptr(u), ctypes.byref(rn), ctypes.byref(fn))
    return code, rn.value, fn.value


def ddel_set_coarse(h, Z, k, flags, on_device):
    """Coarse space: Z holds k vectors over the Gamma DOFs (k x n_gamma, row-major)."""
    return _lib.ddel_set_coarse(h, _ptr(Z), int(k), int(flags), int(on_device))


def ddel_checkpoint_save(h, state, path):
    return _lib.ddel_checkpoint_save(h, ctypes.byref(state), os.fsencode(path))


def ddel_checkpoint_load(h, state, path):
    return _lib.ddel_checkpoint_load(h, ctypes.byref(state), os.fsencode(path))


def ddel_selftest_wait_timeout(poll_limit):
    st = c_int(0)
    code = _lib.ddel_selftest_wait_timeout(int(poll_limit), ctypes.byref(st))
    return code, st.value


def ddel_topopt_step(h, state):
    st = ddel_stats()
    code = _lib.ddel_topopt_step(h, ctypes.byref(state), ctypes.byref(st))
    return code, st


def ddel_batch_solve(handles, us=None, persistent=False):
    """Concurrent solves of several assembled contexts; us: device tensors or
    None; persistent: one persistent launch per batch of iterations
    (ddel_batch_solve_persistent) instead of one stream per problem."""
    n = len(handles)
    harr = (c_void_p * n)(*[h.value if hasattr(h, "value") else h for h in handles])
    uarr = (c_void_p * n)(*[(_ptr(u) if u is not None else None) for u in (us or [None] * n)])
    sts = (ddel_stats * n)()
    fn = _lib.ddel_batch_solve_persistent if persistent else _lib.ddel_batch_solve
    code = fn(harr, n, uarr, sts)
    return code, list(sts)


def ddel_autotune(h, cache_path=None):
    """Times the Schur forms and batch sizes on this GPU; returns (code, mode, check, cached)."""
    m, c, fc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    code = _lib.ddel_autotune(h, cache_path.encode() if cache_path else None, ctypes.byref(m),
                              ctypes.byref(c), ctypes.byref(fc))
    return code, m.value, c.value, bool(fc.value)


def ddel_kernel_info(h):
    k = ddel_kernel_info_t()
    _check(_lib.ddel_kernel_info(h, ctypes.byref(k)), h)
    d = {n: getattr(k, n) for n, _ in k._fields_}
    if k.double_float:
        name = "schur_explicit_df_kernel (FP32-pair arithmetic)"
    elif k.schur_form:
        name = "schur_explicit_kernel<float>" if k.precision else "schur_explicit_f64_kernel"
    else:
        name = "schur2d_kernel" + ("<float>" if k.precision else "<double>")
    d["schur_apply_kernel"] = name
    return d


def ddel_default_gmres_options(**kw):
    o = ddel_gmres_options()
    _lib.ddel_default_gmres_options(ctypes.byref(o))
    _set_fields(o, kw)
    return o


def ddel_gmres_solve(h, opt, f, u, on_device):
    st = ddel_gmres_stats()
    code = _lib.ddel_gmres_solve(h, ctypes.byref(opt), _ptr(f), _ptr(u), on_device, ctypes.byref(st))
    return code, st


def ddel_global_precond_apply(h, opt, r, z, with_record=False):
    """z = S~^-1 r (global form); with_record returns the per-component
    Lanczos record (m, mass iterations, alpha, beta, inner iterations)."""
    rec = np.zeros(3 * (2 + 3 * DDEL_MAX_LANCZOS)) if with_record else None
    code = _lib.ddel_global_precond_apply(h, ctypes.byref(opt), _ptr(r), _ptr(z),
                                          rec.ctypes.data if rec is not None else None)
    if rec is None:
        return code, None
    out = []
    K = DDEL_MAX_LANCZOS
    for c in range(3):
        o = rec[c * (2 + 3 * K):(c + 1) * (2 + 3 * K)]
        m = int(o[0])
        out.append({"m": m, "mass_its": int(o[1]), "alpha": o[2:2 + m].copy(),
                    "beta": o[2 + K:2 + K + max(m - 1, 0)].copy(),
                    "inner_its": o[2 + 2 * K:2 + 2 * K + m].astype(int).tolist()})
    return code, out


def ddel_residual_norm_noalloc(dim, nx, ny, nz, Ke, factors, fixed, f, u, r, norms, stream=None):
    """Residual check that allocates nothing (device tensors in, device norms out)."""
    return _lib.ddel_residual_norm_noalloc(dim, nx, ny, nz, _ptr(Ke), _ptr(factors), _ptr(fixed),
                                           _ptr(f), _ptr(u), _ptr(r), _ptr(norms), stream)


def ddel_gamma_dofs(h, n_gamma):
    out = np.zeros(n_gamma, dtype=np.int64)
    _check(_lib.ddel_gamma_dofs(h, out.ctypes.data), h)
    return out


def ddel_load_vector(h, n_dof):
    out = np.zeros(n_dof)
    _check(_lib.ddel_load_vector(h, out.ctypes.data), h)
    return out


def ddel_fixed_mask(h, n_dof):
    out = np.zeros(n_dof, dtype=np.uint8)
    _check(_lib.ddel_fixed_mask(h, out.ctypes.data), h)
    return out.astype(bool)


# ----------------------------------------------------------------- learned coarse space
DDEL_LEARN_CNN, DDEL_LEARN_HISTORY, DDEL_LEARN_CNN_HISTORY = 0, 1, 2


def ddel_cnn_create(in_ch, out_ch, H, W, max_batch, widths=None, seed=1, stream=None):
    h = c_void_p()
    w = (c_int * 4)(*widths) if widths is not None else None
    code = _lib.ddel_cnn_create(in_ch, out_ch, H, W, max_batch, w, seed, stream, ctypes.byref(h))
    return code, h


ddel_cnn_destroy = _lib.ddel_cnn_destroy


def ddel_cnn_num_params(net):
    return int(_lib.ddel_cnn_num_params(net))


def ddel_cnn_get_params(net, out, on_device):
    return _lib.ddel_cnn_get_params(net, _ptr(out), int(on_device))


def ddel_cnn_set_params(net, p, on_device):
    return _lib.ddel_cnn_set_params(net, _ptr(p), int(on_device))


def ddel_cnn_forward(net, x, n, y):
    return _lib.ddel_cnn_forward(net, _ptr(x), int(n), _ptr(y))


def ddel_cnn_loss_grad(net, x, target, n, grad=None):
    loss = c_double()
    code = _lib.ddel_cnn_loss_grad(net, _ptr(x), _ptr(target), int(n), ctypes.byref(loss), _ptr(grad))
    return code, loss.value


def ddel_cnn_adam_step(net, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    return _lib.ddel_cnn_adam_step(net, lr, beta1, beta2, eps)


def ddel_learner_default_options():
    o = ddel_learner_options()
    _lib.ddel_learner_default_options(ctypes.byref(o))
    return o


def ddel_learner_create(ctx, opt=None):
    h = c_void_p()
    code = _lib.ddel_learner_create(ctx, ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    return code, h


ddel_learner_destroy = _lib.ddel_learner_destroy


def ddel_learner_predict(L, rho_f):
    return _lib.ddel_learner_predict(L, _ptr(rho_f))


def ddel_learner_observe(L, rho_f, u):
    return _lib.ddel_learner_observe(L, _ptr(rho_f), _ptr(u))


def ddel_learner_get_info(L):
    info = ddel_learner_info()
    code = _lib.ddel_learner_get_info(L, ctypes.byref(info))
    return code, info


def ddel_learner_features(L, rho_f, u, x, target):
    return _lib.ddel_learner_features(L, _ptr(rho_f), _ptr(u), _ptr(x), _ptr(target))


def ddel_learner_grid(L):
    H, W = c_int(), c_int()
    code = _lib.ddel_learner_grid(L, ctypes.byref(H), ctypes.byref(W))
    return code, H.value, W.value


def ddel_learner_network(L):
    return _lib.ddel_learner_network(L)


class Learner:
    """Learned (or history) coarse space attached to a Solver; pass it to
    Solver.topopt_state(..., learner=...)."""

    def __init__(self, solver, **options):
        self.opt = ddel_learner_default_options()
        options = dict(options)
        if "widths" in options:
            self.opt.widths = (c_int * 4)(*options.pop("widths"))
        _set_fields(self.opt, options)
        code, self.h = ddel_learner_create(solver.h, self.opt)
        _check(code, solver.h)
        self._solver = solver  # the context must outlive the learner

    def info(self):
        code, info = ddel_learner_get_info(self.h)
        _check(code)
        return info

    def grid(self):
        return ddel_learner_grid(self.h)[1:]

    def close(self):
        if self.h:
            ddel_learner_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- BC marshalling
def node_index(ne, ijk):
    """Global node index of grid node ijk (node-interleaved convention of ddel.h)."""
    n = 0
    for a, x in enumerate(ijk):
        n = n * (ne[a] + 1) + int(x)
    return n


class _BC:
    """Keeps the arrays a ddel_bc points to alive for the duration of create."""

    def __init__(self, ne, spec):
        dim = len(ne)
        self.bc = ddel_bc()
        self.bc.clamp_faces = 0
        for axis, side in spec.get("clamp", []):
            self.bc.clamp_faces |= 1 << (2 * axis + side)
        self.mask = None
        if spec.get("fix"):
            n_dof = dim * int(np.prod([n + 1 for n in ne]))
            self.mask = np.zeros(n_dof, dtype=np.uint8)
            for ijk, c in spec["fix"]:
                self.mask[dim * node_index(ne, ijk) + c] = 1
            self.bc.fixed_dof = self.mask.ctypes.data
        pts = spec.get("point", [])
        self.nodes = np.array([node_index(ne, ijk) for ijk, _ in pts], dtype=np.int64)
        self.forces = np.array([list(fv) for _, fv in pts], dtype=np.float64).reshape(-1)
        self.bc.n_point = len(pts)
        if pts:
            self.bc.point_node = self.nodes.ctypes.data
            self.bc.point_force = self.forces.ctypes.data
        self.bc.traction_face = -1
        if "traction" in spec:
            axis, side, t = spec["traction"]
            self.bc.traction_face = 2 * axis + side
            for k, v in enumerate(t):
                self.bc.traction[k] = v
        for k, v in enumerate(spec.get("body", ())):
            self.bc.body_force[k] = v


class Plan:
    """Host-only set-up (no GPU needed): classification and face operators."""

    def __init__(self, cfg, theta=0.5, plane_stress=True):
        ne = tuple(cfg["ne"])
        self.cfg = cfg
        self.mesh = ddel_mesh(cfg["dim"], ne[0], ne[1], ne[2] if len(ne) > 2 else 0, cfg["sub"])
        self.mat = ddel_material(cfg["E"], cfg["nu"], 1 if plane_stress else 0, cfg["p"], 1e-3)
        bc = _BC(ne, cfg["bc"])
        h = c_void_p()
        _check(_lib.ddel_plan_create(ctypes.byref(self.mesh), ctypes.byref(self.mat),
                                     ctypes.byref(bc.bc), float(theta), ctypes.byref(h)))
        self.h = h
        self.info = ddel_info_t()
        _check(_lib.ddel_plan_info(h, ctypes.byref(self.info)))

    def __del__(self):
        if getattr(self, "h", None):
            _lib.ddel_plan_destroy(self.h)
            self.h = None

    def gamma_dofs(self):
        out = np.zeros(self.info.n_gamma, dtype=np.int64)
        _check(_lib.ddel_plan_gamma_dofs(self.h, out.ctypes.data))
        return out

    def face_block(self, b):
        off, n, hm = ctypes.c_int32(), ctypes.c_int32(), c_double()
        _check(_lib.ddel_plan_face_block(self.h, b, ctypes.byref(off), ctypes.byref(n), None,
                                         ctypes.byref(hm)))
        P = np.zeros((n.value, n.value))
        _check(_lib.ddel_plan_face_block(self.h, b, None, None, P.ctypes.data, None))
        return off.value, n.value, P, hm.value

    def element_matrix(self):
        nd = self.cfg["dim"] * 2 ** self.cfg["dim"]
        K = np.zeros((nd, nd))
        _check(_lib.ddel_plan_element_matrix(self.h, K.ctypes.data))
        return K

    def interface_operator(self, comp):
        """(pos, rowptr, col, M, L): CSR mass and Laplacian on all of Gamma for
        component comp, rows in Gamma order (pos: their Gamma positions)."""
        n, nnz = ctypes.c_int32(), ctypes.c_int64()
        _check(_lib.ddel_plan_interface_operator(self.h, comp, ctypes.byref(n), ctypes.byref(nnz),
                                                 None, None, None, None, None))
        pos = np.zeros(n.value, dtype=np.int32)
        rowptr = np.zeros(n.value + 1, dtype=np.int64)
        col = np.zeros(nnz.value, dtype=np.int32)
        M = np.zeros(nnz.value)
        L = np.zeros(nnz.value)
        _check(_lib.ddel_plan_interface_operator(self.h, comp, ctypes.byref(n), ctypes.byref(nnz),
                                                 pos.ctypes.data, rowptr.ctypes.data, col.ctypes.data,
                                                 M.ctypes.data, L.ctypes.data))
        return pos, rowptr, col, M, L

    def subdomain(self, i):
        ilo = np.zeros(3, dtype=np.int32)
        icnt = np.zeros(3, dtype=np.int32)
        _check(_lib.ddel_plan_subdomain(self.h, i, ilo.ctypes.data, icnt.ctypes.data))
        return ilo, icnt


class Solver:
    """Convenience wrapper: one context for one workload description.

    cfg: dict with dim, ne, sub, E, nu, p, bc (see workloads).  Keyword options
    override ddel_default_options() fields.
    """

    def __init__(self, cfg, stream=None, plane_stress=True, **options):
        ne = tuple(cfg["ne"])
        self.cfg = cfg
        self.mesh = ddel_mesh(cfg["dim"], ne[0], ne[1], ne[2] if len(ne) > 2 else 0, cfg["sub"])
        self.mat = ddel_material(cfg["E"], cfg["nu"], 1 if plane_stress else 0, cfg["p"],
                                 cfg.get("rho_min", 1e-3))
        self.opt = ddel_default_options()
        _set_fields(self.opt, options)
        bc = _BC(ne, cfg["bc"])
        code, self.h = ddel_create(self.mesh, self.mat, bc.bc, self.opt, stream)
        _check(code)
        self.info = ddel_get_info(self.h)

    def close(self):
        if self.h:
            ddel_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, **options):
        _set_fields(self.opt, options)
        _check(ddel_set_options(self.h, self.opt), self.h)

    @property
    def n_dof(self):
        return int(self.info.n_dof)

    @property
    def n_gamma(self):
        return int(self.info.n_gamma)

    def gamma_dofs(self):
        return ddel_gamma_dofs(self.h, self.n_gamma)

    def load_vector(self):
        return ddel_load_vector(self.h, self.n_dof)

    def fixed_mask(self):
        return ddel_fixed_mask(self.h, self.n_dof)

    def assemble(self, rho):
        on_dev = hasattr(rho, "is_cuda") and rho.is_cuda
        if not on_dev:
            rho = np.ascontiguousarray(rho, dtype=np.float64)
        _check(ddel_assemble(self.h, rho, on_dev), self.h)

    def factor(self):
        _check(ddel_factor(self.h), self.h)

    def set_coarse(self, Z, flags=DDEL_COARSE_X0 | DDEL_COARSE_CORRECT):
        """Z: (k, n_gamma) torch CUDA tensor or NumPy array; None or k = 0 removes it."""
        if Z is None:
            _check(ddel_set_coarse(self.h, None, 0, 0, 0), self.h)
            return
        on_dev = hasattr(Z, "is_cuda") and Z.is_cuda
        if not on_dev:
            Z = np.ascontiguousarray(Z, dtype=np.float64)
        self._coarse_ref = Z
        _check(ddel_set_coarse(self.h, Z, Z.shape[0], flags, on_dev), self.h)

    def topopt_state(self, rho, volfrac, r_min=1.5, move=0.2, u=None, rho_phys=None, learner=None,
                     tol_eta=0.0, tol_max=0.0):
        """State for ddel_topopt_step; rho is a CUDA tensor updated in place.
        tol_eta > 0: adaptive analysis tolerance from the last two compliances."""
        ts = ddel_topopt_state()
        ts.rho = _ptr(rho)
        ts.volfrac, ts.r_min, ts.move = volfrac, r_min, move
        ts.tol_eta, ts.tol_max = tol_eta, tol_max
        ts.u = _ptr(u)
        ts.rho_phys = _ptr(rho_phys)
        ts.learner = learner.h.value if learner is not None else None
        self._topo_refs = (rho, u, rho_phys, learner)
        return ts

    def checkpoint_save(self, ts, path):
        _check(ddel_checkpoint_save(self.h, ts, path), self.h)

    def checkpoint_load(self, ts, path):
        _check(ddel_checkpoint_load(self.h, ts, path), self.h)

    def topopt_step(self, ts):
        code, st = ddel_topopt_step(self.h, ts)
        _check(code, self.h)
        return st

    def gmres(self, f=None, u=None, **options):
        """Full-system FGMRES with the block-triangular preconditioner
        (ddel_gmres_solve); options override ddel_default_gmres_options()."""
        on_dev = u is not None and hasattr(u, "is_cuda") and u.is_cuda
        if u is None:
            u = np.zeros(self.n_dof)
        if f is not None and not on_dev:
            f = np.ascontiguousarray(f, dtype=np.float64)
        code, st = ddel_gmres_solve(self.h, ddel_default_gmres_options(**options), f, u, on_dev)
        if code not in (DDEL_OK, DDEL_ENOCONV):
            raise DDELError(code, _lib.ddel_last_error(self.h).decode())
        return u, st

    def solve(self, f=None, u=None, check=True):
        """Solve K u = f; f/u torch CUDA tensors (device path) or NumPy (host path)."""
        on_dev = u is not None and hasattr(u, "is_cuda") and u.is_cuda
        if u is None:
            u = np.zeros(self.n_dof)
        if f is not None and not on_dev:
            f = np.ascontiguousarray(f, dtype=np.float64)
        code, st = ddel_solve(self.h, f, u, on_dev)
        if check and code not in (DDEL_OK,):
            raise DDELError(code, _lib.ddel_last_error(self.h).decode() + f" stats={st.as_dict()}")
        return u, st
