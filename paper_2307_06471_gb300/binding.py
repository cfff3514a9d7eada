"""ctypes binding of the cRKDG C ABI (include/crkdg.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  The functions below carry the ABI's names; ``Solver`` is a thin
object wrapper around one context.  Importing this module does not load the
library; the first call does, and raises if libcrkdg.so is missing -- there
is no fallback implementation.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# CRKDG_LIB may point at another build of the same library (e.g. a variant
# compiled with different launch bounds)
LIB_PATH = os.environ.get("CRKDG_LIB", os.path.join(HERE, "libcrkdg.so"))
MAX_STAGES = 6

OK, EINVAL, ENOMEM, ECUDA, ENONPHYSICAL, ETIMEOUT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
BC_PERIODIC, BC_OUTFLOW, BC_REFLECT, BC_DIRICHLET = 0, 1, 2, 3
FN_CONST, FN_SINE, FN_SINE_PROD, FN_DMR_BOTTOM, FN_DMR_TOP = 0, 1, 2, 3, 4
ADVECTION, EULER = 0, 1
BASIS_P, BASIS_Q = 0, 1
F32, F64, F32C, F32D = 0, 1, 2, 3
LIMIT_FUSED, LIMIT_PASS = 0, 1
MLP_TCGEN05, MLP_MMA_SYNC = 0, 1
FORM_QUADRATURE, FORM_AUTO = 0, 1
FLUX_LLF = 0
ST_NONPHYSICAL, ST_NAN, ST_TIMEOUT = 1, 2, 4


class CrkdgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("crkdg error %d: %s" % (code, msg))
        self.code = code


class Mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("bc", C.c_int * 4), ("bc_fn", C.c_int * 4), ("bc_params", (C.c_double * 16) * 4)]


class Tableau(C.Structure):
    _fields_ = [("s", C.c_int), ("a", C.c_double * (MAX_STAGES * MAX_STAGES)),
                ("b", C.c_double * MAX_STAGES), ("c", C.c_double * MAX_STAGES)]


_lib = None

_SIGS = {
    "crkdg_create": (C.c_int, [C.POINTER(Mesh), C.c_int, C.c_int, C.c_int, C.POINTER(Tableau), C.c_double,
                               C.c_int, C.c_int, C.POINTER(C.c_double), C.c_void_p, C.POINTER(C.c_void_p)]),
    "crkdg_destroy": (None, [C.c_void_p]),
    "crkdg_state_bytes": (C.c_int, [C.POINTER(Mesh), C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
    "crkdg_create_on_buffers": (C.c_int, [C.POINTER(Mesh), C.c_int, C.c_int, C.c_int, C.POINTER(Tableau),
                                          C.c_double, C.c_int, C.c_int, C.POINTER(C.c_double), C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "crkdg_current_state": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_void_p)]),
    "crkdg_sizes": (C.c_int, [C.c_void_p] + [C.POINTER(C.c_int)] * 4),
    "crkdg_quadrature_points": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "crkdg_project_ic": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "crkdg_set_state": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_double]),
    "crkdg_get_state": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "crkdg_cfl_dt": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_double)]),
    "crkdg_step": (C.c_int, [C.c_void_p, C.c_double]),
    "crkdg_advance": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int]),
    "crkdg_run_fixed": (C.c_int, [C.c_void_p, C.c_int, C.c_double]),
    "crkdg_step_device": (C.c_int, [C.c_void_p]),
    "crkdg_rkdg_step": (C.c_int, [C.c_void_p, C.c_double, C.c_int]),
    "crkdg_limit": (C.c_int, [C.c_void_p, C.c_double]),
    "crkdg_positivity": (C.c_int, [C.c_void_p, C.c_double]),
    "crkdg_conservation": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "crkdg_troubled_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_ulonglong)]),
    "crkdg_sync": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint)]),
    "crkdg_time": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "crkdg_set_launch": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "crkdg_get_launch": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "crkdg_set_limit_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "crkdg_run_state_async": (C.c_int, [C.c_void_p, C.c_void_p]),
    "crkdg_step_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_ulonglong)]),
    "crkdg_apply_limit": (C.c_int, [C.c_void_p]),
    "crkdg_set_operator_form": (C.c_int, [C.c_void_p, C.c_int]),
    "crkdg_get_operator_form": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "crkdg_get_limit_mode": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "crkdg_autotune": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "crkdg_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "crkdg_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "crkdg_reduce_state_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                             C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double),
                                             C.c_void_p, C.c_void_p]),
    "crkdg_noalloc_last_error": (C.c_char_p, []),
    "crkdg_alu_peak": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                 C.POINTER(C.c_int)]),
    "crkdg_probe_last_error": (C.c_char_p, []),
    "crkdg_last_error": (C.c_char_p, []),
    "crkdg_version": (C.c_char_p, []),
    "crkdg_batch_create": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int, C.POINTER(Tableau),
                                     C.c_double, C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    "crkdg_batch_destroy": (None, [C.c_void_p]),
    "crkdg_batch_sizes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_longlong), C.POINTER(C.c_int),
                                    C.POINTER(C.c_int)]),
    "crkdg_batch_quadrature_points": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "crkdg_batch_project_ic": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "crkdg_batch_set_state": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_double]),
    "crkdg_batch_get_state": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "crkdg_batch_limit": (C.c_int, [C.c_void_p, C.c_double]),
    "crkdg_batch_positivity": (C.c_int, [C.c_void_p, C.c_double]),
    "crkdg_batch_run": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "crkdg_batch_set_limit_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "crkdg_batch_problem_info": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_ulonglong),
                                           C.POINTER(C.c_uint)]),
    "crkdg_batch_set_launch": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "crkdg_batch_autotune": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_double)]),
    "crkdg_batch_last_error": (C.c_char_p, []),
    "crkdg_batch_features": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_double]),
    "crkdg_mlp_create": (C.c_int, [C.c_ulonglong, C.c_void_p, C.POINTER(C.c_void_p)]),
    "crkdg_mlp_destroy": (None, [C.c_void_p]),
    "crkdg_mlp_n_params": (C.c_int, []),
    "crkdg_mlp_set_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "crkdg_mlp_get_params": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "crkdg_mlp_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                      C.POINTER(C.c_double), C.POINTER(C.c_float)]),
    "crkdg_mlp_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double,
                                  C.c_double, C.c_ulonglong, C.POINTER(C.c_double)]),
    "crkdg_mlp_predict": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "crkdg_mlp_predict_tc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "crkdg_set_indicator_engine": (C.c_int, [C.c_void_p, C.c_int]),
    "crkdg_mlp_last_error": (C.c_char_p, []),
    "crkdg_features": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double]),
    "crkdg_set_indicator": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_double]),
}


class BatchProblem(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double),
                ("y1", C.c_double)]


def lib():
    """Load libcrkdg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libcrkdg.so not built: run paper_2307_06471_gb300.build.build() "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code):
    if code != OK:
        raise CrkdgError(code, lib().crkdg_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


PEAK_F32, PEAK_F32X2, PEAK_F64 = 0, 1, 2


def alu_peak(kind, reps=7, stream=None):
    """(TFLOP/s, median ms per launch, SMs) of the FMA probe crkdg_alu_peak."""
    tf, ms, n = C.c_double(), C.c_double(), C.c_int()
    code = lib().crkdg_alu_peak(int(kind), int(reps), C.c_void_p(stream) if stream else None, C.byref(tf),
                                C.byref(ms), C.byref(n))
    if code != 0:
        raise CrkdgError(code, lib().crkdg_probe_last_error().decode())
    return tf.value, ms.value, n.value


def make_tableau(A, b):
    t = Tableau()
    s = len(b)
    t.s = s
    for i in range(s):
        t.b[i] = b[i]
        t.c[i] = sum(A[i][:i])
        for j in range(s):
            t.a[i * MAX_STAGES + j] = A[i][j]
    return t


def make_mesh(dim, nx, ny, box, bc, bc_fn=(0, 0, 0, 0), bc_params=None):
    m = Mesh()
    m.dim, m.nx, m.ny = dim, nx, ny
    m.x0, m.x1 = box[0], box[1]
    m.y0, m.y1 = (box[2], box[3]) if dim == 2 else (0.0, 1.0)
    for s in range(4):
        m.bc[s] = bc[s]
        m.bc_fn[s] = bc_fn[s]
        if bc_params is not None and bc_params[s] is not None:
            for j, v in enumerate(bc_params[s]):
                m.bc_params[s][j] = float(v)
    return m


def state_bytes(mesh, k, basis, physics, precision):
    """Bytes of one copy of the state (crkdg_state_bytes)."""
    n = C.c_size_t()
    _check(lib().crkdg_state_bytes(C.byref(mesh), int(k), int(basis), int(physics), int(precision), C.byref(n)))
    return n.value


class Solver:
    """One cRKDG context.  State arrays are FP64 numpy planes [v, m, y, x]."""

    def __init__(self, mesh, k, basis, tableau, physics, precision, gamma=1.4, beta=(1.0, 0.0), stream=None,
                 state_buffers=None):
        """state_buffers: None (the context allocates its state) or two
        caller-owned device addresses (ints, e.g. torch data_ptr()) of
        state_bytes(...) bytes each (crkdg_create_on_buffers)."""
        L = lib()
        self.ctx = C.c_void_p()
        pp = np.asarray(beta, dtype=np.float64)
        self._pp = pp
        tab = make_tableau(*tableau) if not isinstance(tableau, Tableau) else tableau
        st = C.c_void_p(stream) if stream else None
        if state_buffers is None:
            _check(L.crkdg_create(C.byref(mesh), k, basis, FLUX_LLF, C.byref(tab), gamma, physics, precision,
                                  _dptr(pp), st, C.byref(self.ctx)))
        else:
            a, b = state_buffers
            _check(L.crkdg_create_on_buffers(C.byref(mesh), k, basis, FLUX_LLF, C.byref(tab), gamma, physics,
                                             precision, _dptr(pp), st, C.c_void_p(int(a)), C.c_void_p(int(b)),
                                             C.byref(self.ctx)))
        self.mesh = mesh
        self.config = {"k": k, "basis": basis, "stages": tab.s, "physics": physics, "precision": precision}
        nc, nm, nv, nq = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(L.crkdg_sizes(self.ctx, C.byref(nc), C.byref(nm), C.byref(nv), C.byref(nq)))
        self.n_cells, self.n_modes, self.n_vars, self.n_qp = nc.value, nm.value, nv.value, nq.value
        self.shape = (self.n_vars, self.n_modes, mesh.ny if mesh.dim == 2 else 1, mesh.nx)

    def close(self):
        if self.ctx:
            lib().crkdg_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def current_state(self):
        """(which copy, device address) of the current state (crkdg_current_state)."""
        w, p = C.c_int(), C.c_void_p()
        _check(lib().crkdg_current_state(self.ctx, C.byref(w), C.byref(p)))
        return w.value, p.value or 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def quadrature_points(self):
        dim = self.mesh.dim
        xy = np.empty(self.n_cells * self.n_qp * dim)
        _check(lib().crkdg_quadrature_points(self.ctx, _dptr(xy)))
        return xy.reshape(self.n_cells, self.n_qp, dim)

    def project_ic(self, values):
        v = np.ascontiguousarray(values, dtype=np.float64).reshape(self.n_cells, self.n_qp, self.n_vars)
        _check(lib().crkdg_project_ic(self.ctx, _dptr(v)))

    def project_function(self, fn):
        """fn(X[, Y]) -> (..., nv) evaluated at the quadrature points."""
        xy = self.quadrature_points()
        if self.mesh.dim == 1:
            vals = fn(xy[..., 0])
        else:
            vals = fn(xy[..., 0], xy[..., 1])
        self.project_ic(np.asarray(vals, dtype=np.float64).reshape(self.n_cells, self.n_qp, self.n_vars))

    def set_state(self, u, t=0.0):
        a = np.ascontiguousarray(u, dtype=np.float64)
        assert a.size == np.prod(self.shape)
        _check(lib().crkdg_set_state(self.ctx, _dptr(a), float(t)))

    def get_state(self, out=None):
        """The FP64 state as a new array, or written into `out` (a C-contiguous
        float64 array of the state's shape, e.g. in pinned host memory)."""
        if out is None:
            out = np.empty(self.shape)
        elif not (out.dtype == np.float64 and out.shape == tuple(self.shape) and out.flags["C_CONTIGUOUS"]):
            raise ValueError("out must be a C-contiguous float64 array of shape %s" % (tuple(self.shape),))
        _check(lib().crkdg_get_state(self.ctx, _dptr(out)))
        return out

    def cfl_dt(self, cfl):
        d = C.c_double()
        _check(lib().crkdg_cfl_dt(self.ctx, cfl, C.byref(d)))
        return d.value

    def step(self, dt):
        _check(lib().crkdg_step(self.ctx, float(dt)))

    def advance(self, n_steps, cfl, t_end, capture=False):
        _check(lib().crkdg_advance(self.ctx, int(n_steps), float(cfl), float(t_end), 1 if capture else 0))

    def rkdg_step(self, dt, order=3):
        _check(lib().crkdg_rkdg_step(self.ctx, float(dt), int(order)))

    def step_device(self):
        _check(lib().crkdg_step_device(self.ctx))

    def run_fixed(self, n_steps, dt):
        _check(lib().crkdg_run_fixed(self.ctx, int(n_steps), float(dt)))

    def limit(self, M):
        _check(lib().crkdg_limit(self.ctx, float(M)))

    def positivity(self, eps):
        _check(lib().crkdg_positivity(self.ctx, float(eps)))

    def conservation(self):
        s = np.empty(self.n_vars)
        _check(lib().crkdg_conservation(self.ctx, _dptr(s)))
        return s

    def troubled_count(self):
        c = C.c_ulonglong()
        _check(lib().crkdg_troubled_count(self.ctx, C.byref(c)))
        return c.value

    def sync(self):
        st = C.c_uint()
        code = lib().crkdg_sync(self.ctx, C.byref(st))
        return code, st.value

    def step_count(self):
        n = C.c_ulonglong()
        _check(lib().crkdg_step_count(self.ctx, C.byref(n)))
        return n.value

    def time(self):
        t = C.c_double()
        _check(lib().crkdg_time(self.ctx, C.byref(t)))
        return t.value

    def set_launch(self, seg_rows=0, warps_per_block=0):
        _check(lib().crkdg_set_launch(self.ctx, int(seg_rows), int(warps_per_block)))

    def set_operator_form(self, form):
        _check(lib().crkdg_set_operator_form(self.ctx, int(form)))

    def get_operator_form(self):
        f = C.c_int()
        _check(lib().crkdg_get_operator_form(self.ctx, C.byref(f)))
        return f.value

    def apply_limit(self):
        _check(lib().crkdg_apply_limit(self.ctx))

    def run_state_async(self, out_ptr):
        """Enqueue a copy of {t, dt, t_end, cfl, max wave speed} into the 5
        doubles at host address out_ptr (pinned memory for an asynchronous
        copy); read them after sync()."""
        _check(lib().crkdg_run_state_async(self.ctx, C.c_void_p(out_ptr)))

    def set_limit_mode(self, mode):
        _check(lib().crkdg_set_limit_mode(self.ctx, int(mode)))

    def set_indicator_engine(self, engine):
        _check(lib().crkdg_set_indicator_engine(self.ctx, int(engine)))

    def get_limit_mode(self):
        m = C.c_int()
        _check(lib().crkdg_get_limit_mode(self.ctx, C.byref(m)))
        return m.value

    def get_launch(self):
        a, b = C.c_int(), C.c_int()
        _check(lib().crkdg_get_launch(self.ctx, C.byref(a), C.byref(b)))
        return a.value, b.value

    def tune_key(self):
        """Key of this solver's launch-tuning entry: mesh size, scheme,
        precision, limit mode and the GPU's name."""
        import torch
        c = self.config
        return "%dx%d/k%d%s/s%d/%s/%s/limit%d/%s" % (
            self.mesh.nx, self.mesh.ny, c["k"], "PQ"[c["basis"]], c["stages"],
            "euler" if c["physics"] == EULER else "advection", ("f32", "f64", "f32c", "f32d")[c["precision"]],
            self.get_limit_mode(), torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu")

    def autotune(self, cache=None):
        """Time the step kernel's launch shapes on the current state and keep
        the fastest (crkdg_autotune); returns microseconds per step kernel.
        cache: path of a JSON file of earlier results, keyed by tune_key();
        a hit applies the stored shape without timing, a miss times and
        stores."""
        import json
        import os
        key = self.tune_key()
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                table = json.load(f)
            if key in table:
                e = table[key]
                self.set_launch(e["seg_rows"], e["warps_per_block"])
                return e["us"]
        us = C.c_double()
        _check(lib().crkdg_autotune(self.ctx, C.byref(us)))
        if cache:
            L, W = self.get_launch()
            table[key] = {"seg_rows": L, "warps_per_block": W, "us": us.value}
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return us.value

    def features(self, X_ptr, y_ptr, M):
        """Features [cells, 40] and TVB labels [cells] into device buffers
        (raw pointers, e.g. torch data_ptr())."""
        _check(lib().crkdg_features(self.ctx, C.c_void_p(X_ptr), C.c_void_p(y_ptr), float(M)))

    def set_indicator(self, net, z_lo=-1.3862943611198906, z_hi=1.3862943611198906):
        _check(lib().crkdg_set_indicator(self.ctx, net.ptr if net is not None else None, float(z_lo), float(z_hi)))

    def save(self, path):
        _check(lib().crkdg_save(self.ctx, path.encode()))

    def load(self, path):
        _check(lib().crkdg_load(self.ctx, path.encode()))


def _bcheck(code):
    if code != OK:
        raise CrkdgError(code, lib().crkdg_batch_last_error().decode())


class Batch:
    """An ensemble of 2D Euler problems advanced together (crkdg_batch_*).
    problems: list of (nx, ny, (x0, x1, y0, y1))."""

    def __init__(self, problems, k, basis, tableau, precision, bc=(BC_OUTFLOW,) * 4, gamma=1.4, stream=None):
        L = lib()
        arr = (BatchProblem * len(problems))()
        for i, (nx, ny, box) in enumerate(problems):
            arr[i] = BatchProblem(nx, ny, box[0], box[1], box[2], box[3])
        self._bc = (C.c_int * 4)(*bc)
        tab = make_tableau(*tableau) if not isinstance(tableau, Tableau) else tableau
        self.ptr = C.c_void_p()
        _bcheck(L.crkdg_batch_create(C.cast(arr, C.c_void_p), len(problems), self._bc, k, basis, C.byref(tab), gamma,
                                     precision, C.c_void_p(stream) if stream else None, C.byref(self.ptr)))
        self.problems = problems
        self.k = k
        n, nm, nt = C.c_int(), C.c_int(), C.c_int()
        cells = C.c_longlong()
        _bcheck(L.crkdg_batch_sizes(self.ptr, C.byref(n), C.byref(cells), C.byref(nm), C.byref(nt)))
        self.n, self.total_cells, self.n_modes, self.n_tasks = n.value, cells.value, nm.value, nt.value

    def close(self):
        if self.ptr:
            lib().crkdg_batch_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def quadrature_points(self, p):
        nx, ny, _ = self.problems[p]
        nq = (self.k + 1) ** 2
        xy = np.empty(nx * ny * nq * 2)
        _bcheck(lib().crkdg_batch_quadrature_points(self.ptr, p, _dptr(xy)))
        return xy.reshape(nx * ny, nq, 2)

    def project_function(self, p, fn):
        xy = self.quadrature_points(p)
        vals = np.ascontiguousarray(fn(xy[..., 0], xy[..., 1]), dtype=np.float64)
        _bcheck(lib().crkdg_batch_project_ic(self.ptr, p, _dptr(vals)))

    def set_state(self, p, u, t=0.0):
        a = np.ascontiguousarray(u, dtype=np.float64)
        _bcheck(lib().crkdg_batch_set_state(self.ptr, p, _dptr(a), float(t)))

    def get_state(self, p):
        nx, ny, _ = self.problems[p]
        a = np.empty((4, self.n_modes, ny, nx))
        _bcheck(lib().crkdg_batch_get_state(self.ptr, p, _dptr(a)))
        return a

    def set_limit_mode(self, mode):
        _bcheck(lib().crkdg_batch_set_limit_mode(self.ptr, int(mode)))

    def limit(self, M):
        _bcheck(lib().crkdg_batch_limit(self.ptr, float(M)))

    def positivity(self, eps):
        _bcheck(lib().crkdg_batch_positivity(self.ptr, float(eps)))

    def run(self, cfl, t_end, steps_per_graph=8, max_graphs=1):
        d = C.c_int()
        _bcheck(lib().crkdg_batch_run(self.ptr, float(cfl), float(t_end), int(steps_per_graph), int(max_graphs),
                                      C.byref(d)))
        return d.value

    def info(self, p):
        t, st = C.c_double(), C.c_uint()
        n = C.c_ulonglong()
        _bcheck(lib().crkdg_batch_problem_info(self.ptr, p, C.byref(t), C.byref(n), C.byref(st)))
        return t.value, n.value, st.value

    def set_launch(self, seg_rows=0, warps_per_block=0):
        _bcheck(lib().crkdg_batch_set_launch(self.ptr, int(seg_rows), int(warps_per_block)))

    def autotune(self, cfl):
        us = C.c_double()
        _bcheck(lib().crkdg_batch_autotune(self.ptr, float(cfl), C.byref(us)))
        return us.value

    def features(self, p, X_ptr, y_ptr, M):
        _bcheck(lib().crkdg_batch_features(self.ptr, p, C.c_void_p(X_ptr), C.c_void_p(y_ptr), float(M)))


def _mcheck(code):
    if code != OK:
        raise CrkdgError(code, lib().crkdg_mlp_last_error().decode())


class MLP:
    """The learned troubled-cell indicator network (crkdg_mlp_*).  X/y/logit
    arguments are device pointers (e.g. torch tensors' data_ptr())."""

    def __init__(self, seed=0, stream=None):
        self.ptr = C.c_void_p()
        _mcheck(lib().crkdg_mlp_create(seed, C.c_void_p(stream) if stream else None, C.byref(self.ptr)))
        self.n_params = lib().crkdg_mlp_n_params()

    def close(self):
        if self.ptr:
            lib().crkdg_mlp_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        a = np.empty(self.n_params, dtype=np.float32)
        _mcheck(lib().crkdg_mlp_get_params(self.ptr, a.ctypes.data_as(C.POINTER(C.c_float))))
        return a

    def set_params(self, a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        assert a.size == self.n_params
        _mcheck(lib().crkdg_mlp_set_params(self.ptr, a.ctypes.data_as(C.POINTER(C.c_float))))

    def loss_grad(self, X_ptr, y_ptr, n, pos_weight=1.0):
        loss = C.c_double()
        g = np.empty(self.n_params, dtype=np.float32)
        _mcheck(lib().crkdg_mlp_loss_grad(self.ptr, C.c_void_p(X_ptr), C.c_void_p(y_ptr), int(n), float(pos_weight),
                                          C.byref(loss), g.ctypes.data_as(C.POINTER(C.c_float))))
        return loss.value, g

    def train(self, X_ptr, y_ptr, n, epochs, batch, lr, pos_weight=1.0, seed=0):
        loss = C.c_double()
        _mcheck(lib().crkdg_mlp_train(self.ptr, C.c_void_p(X_ptr), C.c_void_p(y_ptr), int(n), int(epochs), int(batch),
                                      float(lr), float(pos_weight), seed, C.byref(loss)))
        return loss.value

    def predict(self, X_ptr, n, out_ptr):
        _mcheck(lib().crkdg_mlp_predict(self.ptr, C.c_void_p(X_ptr), int(n), C.c_void_p(out_ptr)))

    def predict_tc(self, X_ptr, n, out_ptr):
        """The logits on the tcgen05 tensor cores (tiles of 512 samples)."""
        _mcheck(lib().crkdg_mlp_predict_tc(self.ptr, C.c_void_p(X_ptr), int(n), C.c_void_p(out_ptr)))
