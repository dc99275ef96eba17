"""ctypes binding of libpff (C ABI in include/pff.h).  Argument marshalling only.

Every function of the C ABI is exposed under the same name without the
``pff_`` prefix (``create_problem``, ``set_modulus_field``, ``set_model``,
``step_load``, ``get_fields``, ...), plus small ``Problem`` / ``Batch``
wrappers.  Host arrays are NumPy FP64; a CUDA ``torch.Tensor`` (FP64) is
passed as a device pointer.  Importing this module loads ``libpff.so`` and
raises ImportError when it is missing: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libpff.so")
if not os.path.exists(_LIBPATH):
    raise ImportError(f"libpff.so not found at {_LIBPATH}; build it with __graft_entry__.build() "
                      "(needs nvcc; the library only runs on an sm_103a GPU)")
lib = ctypes.CDLL(_LIBPATH)

OK, ERR_INVALID_ARG, ERR_OOM, ERR_NOT_CONVERGED, ERR_BARRIER_TIMEOUT, ERR_CUDA, ERR_STATE = 0, -1, -2, -3, -4, -5, -6
FP64, MIXED = 0, 1
AT1, AT2 = 1, 2
ISOTROPIC, SPECTRAL, SPECTRAL_STRESSFREE, VOLDEV, SPECTRAL_VOLDEV = 0, 1, 2, 3, 4
CRACK_SET, DAMAGE = 0, 1
NEAR_EQUILIBRIUM, ALTERNATING_MIN, TIME_DEPENDENT = 0, 1, 2
FIELD_STRAIN, FIELD_EPS_STAR, FIELD_STRESS, FIELD_PHI, FIELD_PSI_PLUS, FIELD_DRIVING_FORCE, \
    FIELD_MODULUS, FIELD_ACTIVE, FIELD_UPDATE = range(9)
_TENSOR_FIELDS = {FIELD_STRAIN, FIELD_EPS_STAR, FIELD_STRESS}
CRACK_SEGMENT, CRACK_EDGE = 0, 1
IC_PHASE_FIELD, IC_MODULUS = 0, 1
MICRO_RANDOM, MICRO_TWO_PHASE = 0, 1


class Params(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("Gc", ctypes.c_double), ("ell", ctypes.c_double), ("dx", ctypes.c_double),
                ("mech_tol", ctypes.c_double), ("mech_cg_rtol", ctypes.c_double),
                ("mech_max_newton", ctypes.c_int), ("mech_max_cg", ctypes.c_int),
                ("pf_tol", ctypes.c_double), ("pf_atol", ctypes.c_double), ("pf_max_iter", ctypes.c_int),
                ("eta_over_dt", ctypes.c_double), ("F_max", ctypes.c_double), ("thresh", ctypes.c_double),
                ("dphi_min", ctypes.c_double), ("C_broken", ctypes.c_double),
                ("crack_set_threshold", ctypes.c_double), ("d_eps_bar", ctypes.c_double * 3),
                ("compute_energies", ctypes.c_int), ("evolution", ctypes.c_int), ("tol_am", ctypes.c_double),
                ("am_max_inner", ctypes.c_int), ("dt_min", ctypes.c_double), ("dt_max", ctypes.c_double),
                ("dphi_max", ctypes.c_double), ("pf_precondition", ctypes.c_int)]


class StepReport(ctypes.Structure):
    _fields_ = [("eps_bar", ctypes.c_double * 3), ("sig_bar", ctypes.c_double * 3), ("C_bar", ctypes.c_double),
                ("gamma", ctypes.c_double), ("dphi_L1", ctypes.c_double), ("F_e", ctypes.c_double),
                ("F_f", ctypes.c_double), ("mF_max", ctypes.c_double), ("D_max", ctypes.c_double),
                ("mech_res", ctypes.c_double), ("pf_res", ctypes.c_double),
                ("rescaled", ctypes.c_int), ("incremented", ctypes.c_int), ("newton_iters", ctypes.c_int),
                ("mech_cg_iters", ctypes.c_int), ("bccg_iters", ctypes.c_int), ("n_active", ctypes.c_int),
                ("istar", ctypes.c_int), ("broken", ctypes.c_int), ("status", ctypes.c_int),
                ("bccg_clamp_iters", ctypes.c_int), ("dt", ctypes.c_double), ("inner_iters", ctypes.c_int),
                ("bccg_full_iters", ctypes.c_int)]

    def to_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


class MicroParams(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("L_cut", ctypes.c_double), ("std_target", ctypes.c_double),
                ("xi_min", ctypes.c_double), ("a", ctypes.c_double), ("ac_iters", ctypes.c_int),
                ("E0", ctypes.c_double)]


_P = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)
_SIGS = {
    "pff_default_params": (ctypes.c_int, [ctypes.POINTER(Params)]),
    "pff_create_problem": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "pff_destroy_problem": (ctypes.c_int, [_P]),
    "pff_last_error": (ctypes.c_char_p, [_P]),
    "pff_problem_info": (ctypes.c_int, [_P, _IP, _IP, _IP]),
    "pff_problem_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "pff_set_params": (ctypes.c_int, [_P, ctypes.POINTER(Params)]),
    "pff_get_params": (ctypes.c_int, [_P, ctypes.POINTER(Params)]),
    "pff_set_model": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "pff_set_modulus_field": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "pff_set_phase_field": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "pff_set_strain": (ctypes.c_int, [_P, _P, _DP, ctypes.c_int]),
    "pff_init_crack": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double]),
    "pff_default_micro_params": (ctypes.c_int, [ctypes.POINTER(MicroParams)]),
    "pff_generate_modulus": (ctypes.c_int, [_P, ctypes.POINTER(MicroParams), _P, ctypes.c_int]),
    "pff_set_flag": (ctypes.c_int, [_P, ctypes.c_int]),
    "pff_step_load": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(StepReport), _IP]),
    "pff_solve_mechanics": (ctypes.c_int, [_P, ctypes.POINTER(StepReport)]),
    "pff_solve_phase_field": (ctypes.c_int, [_P, ctypes.POINTER(StepReport)]),
    "pff_get_fields": (ctypes.c_int, [_P, ctypes.c_int, _DP]),
    "pff_get_device_ptr": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P), _IP]),
    "pff_apply_projection": (ctypes.c_int, [_P, _DP, _DP]),
    "pff_apply_laplacian": (ctypes.c_int, [_P, _DP, _DP]),
    "pff_constitutive": (ctypes.c_int, [_P, _DP, _DP, _DP, _DP, _DP, _DP]),
    "pff_create_batch": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    "pff_destroy_batch": (ctypes.c_int, [_P]),
    "pff_batch_admit": (ctypes.c_int, [_P, _P, _IP]),
    "pff_batch_release": (ctypes.c_int, [_P, ctypes.c_int]),
    "pff_batch_step": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(StepReport), _IP]),
    "pff_batch_set_group_size": (ctypes.c_int, [_P, ctypes.c_int]),
    "pff_batch_autotune": (ctypes.c_int, [_P, _IP, ctypes.c_int, ctypes.c_int, _IP, ctypes.POINTER(StepReport), _IP]),
    "pff_set_kernel_variant": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "pff_get_kernel_variant": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _IP]),
    "pff_batch_autotune_kernels": (ctypes.c_int, [_P, ctypes.c_int, _IP, _DP, ctypes.POINTER(StepReport), _IP]),
    "pff_kernel_launches": (ctypes.c_ulonglong, []),
    "pff_timing_enable": (ctypes.c_int, [ctypes.c_int]),
    "pff_set_graphs": (ctypes.c_int, [ctypes.c_int]),
    "pff_set_pdl": (ctypes.c_int, [ctypes.c_int]),
    "pff_set_persistent": (ctypes.c_int, [ctypes.c_int]),
    "pff_set_barrier_spin_limit": (ctypes.c_int, [ctypes.c_longlong]),
    "pff_set_cluster_mechanics": (ctypes.c_int, [ctypes.c_int]),
    "pff_apply_laplacian_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, _P, _P, _P,
                                                   ctypes.POINTER(ctypes.c_char_p)]),
    "pff_apply_laplacian_noalloc_f32": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, _P, _P, _P,
                                                       ctypes.POINTER(ctypes.c_char_p)]),
    "pff_timing_reset": (ctypes.c_int, []),
    "pff_timing_read": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _DP, ctypes.POINTER(ctypes.c_ulonglong)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class PffError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libpff error {code}: {msg}")
        self.code = code


def _check(rc, h=None, allow=()):
    if rc != OK and rc not in allow:
        msg = lib.pff_last_error(h).decode() if h else ""
        raise PffError(rc, msg)
    return rc


def _dptr(a):
    return a.ctypes.data_as(_DP) if a is not None else None


def _as_host(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _field_arg(a, n):
    """(pointer, on_device, keepalive) for a NumPy array or a CUDA torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != n:
                raise ValueError("device fields must be contiguous float64 tensors of the grid size")
            if a.is_cuda:
                return ctypes.c_void_p(a.data_ptr()), 1, a
            a = a.numpy()
    except ImportError:
        pass
    h = _as_host(a, n)
    return h.ctypes.data_as(ctypes.c_void_p), 0, h


# ---------------------------------------------------------------------------- C-named functions
def default_params():
    p = Params()
    _check(lib.pff_default_params(ctypes.byref(p)))
    return p


def problem_bytes(nx, ny, precision):
    return int(lib.pff_problem_bytes(nx, ny, precision))


def kernel_launches():
    return int(lib.pff_kernel_launches())


def set_persistent(on=True):
    return _check(lib.pff_set_persistent(1 if on else 0))


def set_cluster_mechanics(on=True):
    """Mechanics solves of FP32 512^2 problems in one cluster launch (True) or per kernel (False, default)."""
    return _check(lib.pff_set_cluster_mechanics(1 if on else 0))


def set_barrier_spin_limit(cycles=0):
    """Wait limit (clock cycles) of the persistent solve's grid barriers; 0: default."""
    return _check(lib.pff_set_barrier_spin_limit(int(cycles)))


def set_pdl(on=True):
    return _check(lib.pff_set_pdl(1 if on else 0))


def set_graphs(on=True):
    """True/1: plain graphs; 2: graphs with conditional nodes; False/0: direct launches."""
    return _check(lib.pff_set_graphs(int(on)))


def timing_enable(on=True):
    return _check(lib.pff_timing_enable(1 if on else 0))


def timing_reset():
    return _check(lib.pff_timing_reset())


def timing_read(family, op):
    """(total device ms, launches) of one kernel class since the last reset."""
    ms = ctypes.c_double()
    n = ctypes.c_ulonglong()
    _check(lib.pff_timing_read(family, op, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, int(n.value)


def create_problem(nx, ny, precision=MIXED, stream=None):
    h = _P()
    st = ctypes.c_void_p(stream) if stream else None
    _check(lib.pff_create_problem(nx, ny, precision, st, ctypes.byref(h)))
    return h


def destroy_problem(h):
    return _check(lib.pff_destroy_problem(h))


_PARAM_FIELDS = frozenset(f[0] for f in Params._fields_)


def set_params(h, p):
    return _check(lib.pff_set_params(h, ctypes.byref(p)), h)


def get_params(h):
    p = Params()
    _check(lib.pff_get_params(h, ctypes.byref(p)), h)
    return p


def set_model(h, fracture, split, irreversibility):
    return _check(lib.pff_set_model(h, fracture, split, irreversibility), h)


def _nxny(h):
    nx, ny, pr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib.pff_problem_info(h, ctypes.byref(nx), ctypes.byref(ny), ctypes.byref(pr)), h)
    return nx.value, ny.value, pr.value


def problem_info(h):
    return _nxny(h)


def set_modulus_field(h, E):
    nx, ny, _ = _nxny(h)
    ptr, dev, keep = _field_arg(E, nx * ny)
    return _check(lib.pff_set_modulus_field(h, ptr, dev), h)


def set_phase_field(h, phi):
    nx, ny, _ = _nxny(h)
    ptr, dev, keep = _field_arg(phi, nx * ny)
    return _check(lib.pff_set_phase_field(h, ptr, dev), h)


def init_crack(h, target=IC_PHASE_FIELD, shape=CRACK_SEGMENT, xc=0.0, yc=0.0, length=0.0, E0=1.0):
    return _check(lib.pff_init_crack(h, int(target), int(shape), float(xc), float(yc), float(length), float(E0)), h)


def default_micro_params(**kw):
    mp = MicroParams()
    _check(lib.pff_default_micro_params(ctypes.byref(mp)))
    for k, v in kw.items():
        if not hasattr(mp, k):
            raise AttributeError(k)
        setattr(mp, k, v)
    return mp


def generate_modulus(h, noise, kind=MICRO_RANDOM, **kw):
    """E = E0 xi from the white noise field (host array or CUDA FP64 tensor) by the
    Sec. 3.3 generator of the given kind; keyword arguments override pff_micro_params."""
    nx, ny, _ = _nxny(h)
    mp = default_micro_params(kind=int(kind), **kw)
    ptr, dev, keep = _field_arg(noise, nx * ny)
    return _check(lib.pff_generate_modulus(h, ctypes.byref(mp), ptr, dev), h)


def set_strain(h, eps_star, eps_bar):
    nx, ny, _ = _nxny(h)
    eb = (ctypes.c_double * 3)(*[float(x) for x in eps_bar])
    if eps_star is None:
        return _check(lib.pff_set_strain(h, None, eb, 0), h)
    ptr, dev, keep = _field_arg(eps_star, 3 * nx * ny)
    return _check(lib.pff_set_strain(h, ptr, eb, dev), h)


def set_flag(h, flag):
    return _check(lib.pff_set_flag(h, int(flag)), h)


def step_load(h, n_steps=1, allow_not_converged=True):
    reps = (StepReport * max(1, n_steps))()
    done = ctypes.c_int()
    _check(lib.pff_step_load(h, n_steps, reps, ctypes.byref(done)), h,
           allow=(ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return [reps[i].to_dict() for i in range(done.value)]


def solve_mechanics(h):
    r = StepReport()
    _check(lib.pff_solve_mechanics(h, ctypes.byref(r)), h, allow=(ERR_NOT_CONVERGED,))
    return r.to_dict()


def solve_phase_field(h):
    r = StepReport()
    _check(lib.pff_solve_phase_field(h, ctypes.byref(r)), h, allow=(ERR_NOT_CONVERGED,))
    return r.to_dict()


def get_fields(h, which, out=None):
    """FP64 copy of a field; out: a C-contiguous float64 array of the field's size to fill
    (for example one backed by pinned memory), else a new array."""
    nx, ny, _ = _nxny(h)
    ncomp = 3 if which in _TENSOR_FIELDS else 1
    if out is None:
        out = np.empty(ncomp * nx * ny, dtype=np.float64)
    elif out.dtype != np.float64 or out.size != ncomp * nx * ny or not out.flags.c_contiguous:
        raise ValueError(f"out must be a C-contiguous float64 array of {ncomp * nx * ny} values")
    _check(lib.pff_get_fields(h, which, _dptr(out)), h)
    return out.reshape((3, ny, nx) if ncomp == 3 else (ny, nx))


def get_device_ptr(h, which):
    p = _P()
    dt = ctypes.c_int()
    _check(lib.pff_get_device_ptr(h, which, ctypes.byref(p), ctypes.byref(dt)), h)
    return p.value, dt.value


def apply_projection(h, field3):
    nx, ny, _ = _nxny(h)
    a = _as_host(field3, 3 * nx * ny)
    out = np.empty(3 * nx * ny)
    _check(lib.pff_apply_projection(h, _dptr(a), _dptr(out)), h)
    return out.reshape(3, ny, nx)


def apply_laplacian(h, field):
    nx, ny, _ = _nxny(h)
    a = _as_host(field, nx * ny)
    out = np.empty(nx * ny)
    _check(lib.pff_apply_laplacian(h, _dptr(a), _dptr(out)), h)
    return out.reshape(ny, nx)


def constitutive(h, eps3, phi, p3=None):
    """Returns (sigma (3,ny,nx), psi_0^+ (ny,nx), C:p (3,ny,nx) or None)."""
    nx, ny, _ = _nxny(h)
    n = nx * ny
    e = _as_host(eps3, 3 * n)
    ph = _as_host(phi, n)
    pp = _as_host(p3, 3 * n) if p3 is not None else None
    sig = np.empty(3 * n)
    psi = np.empty(n)
    tang = np.empty(3 * n) if p3 is not None else None
    _check(lib.pff_constitutive(h, _dptr(e), _dptr(ph), _dptr(pp), _dptr(sig), _dptr(psi), _dptr(tang)), h)
    return sig.reshape(3, ny, nx), psi.reshape(ny, nx), (tang.reshape(3, ny, nx) if tang is not None else None)


def create_batch(max_slots, hbm_budget, stream=None):
    b = _P()
    _check(lib.pff_create_batch(max_slots, hbm_budget, ctypes.c_void_p(stream) if stream else None, ctypes.byref(b)))
    return b


def destroy_batch(b):
    return _check(lib.pff_destroy_batch(b))


def batch_admit(b, h):
    """Returns the slot index, or None when the problem does not fit (OOM) or no slot is free."""
    s = ctypes.c_int(-1)
    rc = lib.pff_batch_admit(b, h, ctypes.byref(s))
    if rc in (ERR_OOM, ERR_STATE):
        return None
    _check(rc)
    return s.value


def batch_set_group_size(b, n):
    return _check(lib.pff_batch_set_group_size(b, int(n)))


def batch_release(b, slot):
    return _check(lib.pff_batch_release(b, slot))


def batch_step(b, max_slots, n_steps=1):
    reps = (StepReport * (max_slots * max(1, n_steps)))()
    done = (ctypes.c_int * max_slots)()
    _check(lib.pff_batch_step(b, n_steps, reps, done), allow=(ERR_NOT_CONVERGED,))
    return [[reps[i * n_steps + s].to_dict() for s in range(done[i])] for i in range(max_slots)]


def batch_autotune(b, max_slots, group_sizes=(1, 2, 4, 8), steps_each=2):
    """Measure each launch grouping on real load steps and keep the fastest; returns
    (chosen group size, per-slot lists of the step reports of the steps run)."""
    n = len(group_sizes)
    total = n * (steps_each + 1)
    gs = (ctypes.c_int * n)(*[int(g) for g in group_sizes])
    reps = (StepReport * (max_slots * total))()
    done = (ctypes.c_int * max_slots)()
    chosen = ctypes.c_int()
    _check(lib.pff_batch_autotune(b, gs, n, steps_each, ctypes.byref(chosen), reps, done), allow=(ERR_NOT_CONVERGED,))
    return chosen.value, [[reps[i * total + s].to_dict() for s in range(done[i])] for i in range(max_slots)]


VARIANT_COLUMN_SHAPE, VARIANT_BCCG_PASSES = 2, 3


def set_kernel_variant(kind, grid_n, ncomp, variant):
    return _check(lib.pff_set_kernel_variant(kind, grid_n, ncomp, variant))


def get_kernel_variant(kind, grid_n, ncomp):
    v = ctypes.c_int()
    _check(lib.pff_get_kernel_variant(kind, grid_n, ncomp, ctypes.byref(v)))
    return v.value


def batch_autotune_kernels(b, max_slots, steps_each=2):
    """Measure the eight kernel-variant combinations on load steps of the batch and keep the
    fastest; returns ((1-component column shape, 3-component column shape, BCCG passes),
    scores, per-slot step reports)."""
    total = 16 * steps_each
    chosen = (ctypes.c_int * 3)()
    scores = (ctypes.c_double * 8)()
    reps = (StepReport * (max_slots * total))()
    done = (ctypes.c_int * max_slots)()
    _check(lib.pff_batch_autotune_kernels(b, steps_each, chosen, scores, reps, done), allow=(ERR_NOT_CONVERGED,))
    return ((chosen[0], chosen[1], chosen[2]), list(scores),
            [[reps[i * total + s].to_dict() for s in range(done[i])] for i in range(max_slots)])


# ---------------------------------------------------------------------------- convenience wrappers
_MODEL = {"AT1": AT1, "AT2": AT2, "ISOTROPIC": ISOTROPIC, "SPECTRAL": SPECTRAL,
          "SPECTRAL_STRESSFREE": SPECTRAL_STRESSFREE, "VOLDEV": VOLDEV, "SPECTRAL_VOLDEV": SPECTRAL_VOLDEV,
          "CRACK_SET": CRACK_SET, "DAMAGE": DAMAGE, "NEAR_EQUILIBRIUM": NEAR_EQUILIBRIUM,
          "ALTERNATING_MIN": ALTERNATING_MIN, "TIME_DEPENDENT": TIME_DEPENDENT}


class Problem:
    """Owning handle of one problem (destroyed with the object or by close())."""

    def __init__(self, nx, ny, precision=MIXED, stream=None, E=None, params=None, model=None):
        self.nx, self.ny, self.precision = nx, ny, precision
        self.h = create_problem(nx, ny, precision, stream)
        if params:
            self.set_params(**params)
        if model:
            self.set_model(*model)
        if E is not None:
            set_modulus_field(self.h, E)

    def close(self):
        if getattr(self, "h", None):
            destroy_problem(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, **kw):
        p = get_params(self.h)
        for k, v in kw.items():
            if k == "d_eps_bar":
                for j in range(3):
                    p.d_eps_bar[j] = float(v[j])
            elif k in _PARAM_FIELDS:
                setattr(p, k, v)
            else:
                raise TypeError(f"unknown parameter {k!r}")
        set_params(self.h, p)

    def set_model(self, fracture, split, irreversibility):
        f = _MODEL.get(fracture, fracture)
        s = _MODEL.get(split, split)
        i = _MODEL.get(irreversibility, irreversibility)
        set_model(self.h, f, s, i)

    def __getattr__(self, name):
        fn = globals().get(name)
        if callable(fn) and name in ("set_modulus_field", "set_phase_field", "set_strain", "set_flag", "step_load",
                                     "init_crack", "generate_modulus",
                                     "solve_mechanics", "solve_phase_field", "get_fields", "get_device_ptr",
                                     "apply_projection", "apply_laplacian", "constitutive", "get_params"):
            return lambda *a, **k: fn(self.h, *a, **k)
        raise AttributeError(name)
