"""GB300 Newton-GMRES-BDDC tangent solver for cardiac mechanics.

Thin Python binding over the C ABI of ``include/cardiac_bddc.h``
(libcardiac_bddc.so, built in-tree for sm_103a).  This module only
marshals arguments: every step of the solve runs in the library's CUDA
kernels.  Device vectors are ``torch`` FP64 CUDA tensors; the current torch
stream is passed as the CUDA stream.

Importing the package does not require a GPU, but it does require the
compiled library; ``build()`` compiles it.  There is no CPU fallback.
"""
import ctypes
import os

import numpy as np

from . import _build

__all__ = [
    "build", "load_library", "Problem", "BDDC", "SolveOptions", "CBDDCError",
    "FP64", "FP32", "SCALING_COUNTING", "SCALING_DELUXE", "scaling_code",
    "COARSE_GALERKIN", "COARSE_PETROV", "coarse_code",
    "PRIMAL_V", "PRIMAL_E", "PRIMAL_F", "PRIMAL_R", "primal_mask",
    "EXPORTED_SYMBOLS",
]

OK, EINVAL, ECUDA, EPIVOT, EINVERTED, ENOCONV, ETIMEOUT, ENOMEM = range(8)
HEX_Q1, HEX_Q2, TET_P1, TET_P2 = 1, 2, 3, 4
FIBER_SLAB_HELIX, FIBER_NODAL = 1, 2
FP64, FP32 = 0, 1
SCALING_COUNTING, SCALING_DELUXE = 0, 1
COARSE_GALERKIN, COARSE_PETROV = 0, 1
PRIMAL_V, PRIMAL_E, PRIMAL_F, PRIMAL_R = 1, 2, 4, 8
MAX_RECORDS = 512

EXPORTED_SYMBOLS = [
    "fem_problem_create", "fem_problem_destroy", "fem_problem_get_info",
    "fem_residual", "fem_assemble_tangent", "fem_tangent_copy", "fem_spmv", "fem_set_time_state",
    "bddc_setup", "bddc_apply", "bddc_apply_noalloc", "bddc_destroy", "bddc_get_info",
    "gmres_solve", "newton_step", "newton_step_host", "newton_gmres_solve",
    "cbddc_kernel_launches", "cbddc_timer_start", "cbddc_timer_stop",
    "cbddc_set_tensor_cores", "cbddc_timer_enable", "cbddc_timer_result", "cbddc_last_error",
]
(TIMER_OFF, TIMER_SWEEP_GEMM, TIMER_ELEMENT, TIMER_APPLY, TIMER_SPMV, TIMER_ORTH, TIMER_SETUP,
 TIMER_LEVEL2_SETUP, TIMER_LEVEL2_APPLY, TIMER_COARSE_SETUP, TIMER_COARSE_APPLY,
 TIMER_SETUP_GEMM_F64) = range(12)


def primal_mask(spec):
    """'V', 'VE', 'VEF', 'EF', 'VER', ... -> bit mask (R: rotations of the
    edge and face classes)."""
    m = 0
    for ch in spec:
        m |= {"V": PRIMAL_V, "E": PRIMAL_E, "F": PRIMAL_F, "R": PRIMAL_R}[ch]
    return m


def scaling_code(spec):
    """'counting' / 'deluxe' (or the code itself) -> CBDDC_SCALING_* code."""
    if isinstance(spec, int):
        return spec
    return {"counting": SCALING_COUNTING, "deluxe": SCALING_DELUXE}[spec]


def coarse_code(spec):
    """'galerkin' / 'petrov' (or the code itself) -> CBDDC_COARSE_* code."""
    if isinstance(spec, int):
        return spec
    return {"galerkin": COARSE_GALERKIN, "petrov": COARSE_PETROV}[spec]


class CBDDCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("cardiac_bddc error %d: %s" % (code, msg))
        self.code = code


_i32p = ctypes.POINTER(ctypes.c_int32)
_dp = ctypes.POINTER(ctypes.c_double)


class _Desc(ctypes.Structure):
    _fields_ = [
        ("elem_type", ctypes.c_int), ("n_nodes", ctypes.c_int), ("coords", _dp),
        ("n_elems", ctypes.c_int), ("elems", _i32p), ("elem_part", _i32p),
        ("n_parts", ctypes.c_int), ("n_dirichlet", ctypes.c_int), ("dirichlet_nodes", _i32p),
        ("n_pressure_faces", ctypes.c_int), ("pressure_faces", _i32p),
        ("fiber_kind", ctypes.c_int), ("fiber_params", ctypes.c_double * 8),
        ("material", ctypes.c_double * 8), ("pressure", ctypes.c_double),
        ("gamma", ctypes.c_double), ("fiber_nodal", _dp),
        ("rho", ctypes.c_double), ("n_robin_faces", ctypes.c_int), ("robin_faces", _i32p),
        ("robin", (ctypes.c_double * 4) * 2),
    ]


class _ProblemInfo(ctypes.Structure):
    _fields_ = [
        ("n_free", ctypes.c_int64), ("n_block_rows", ctypes.c_int64), ("nnzb", ctypes.c_int64),
        ("n_parts", ctypes.c_int), ("n_vertices", ctypes.c_int), ("n_edges", ctypes.c_int),
        ("n_faces", ctypes.c_int), ("max_local_dofs", ctypes.c_int64),
        ("sum_local_dofs", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
    ]


class _Tangent(ctypes.Structure):
    _fields_ = [("vals", ctypes.c_void_p), ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p),
                ("n_block_rows", ctypes.c_int64), ("nnzb", ctypes.c_int64)]


class _BddcOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("primal", ctypes.c_int), ("pivot_tol", ctypes.c_double),
                ("levels", ctypes.c_int), ("n_parts2", ctypes.c_int), ("part2", _i32p),
                ("primal2", ctypes.c_int), ("precision2", ctypes.c_int), ("scaling", ctypes.c_int),
                ("coarse", ctypes.c_int), ("sweep_block", ctypes.c_int), ("tile_order", ctypes.c_int)]


class _BddcInfo(ctypes.Structure):
    _fields_ = [("n_primal", ctypes.c_int), ("n_primal2", ctypes.c_int), ("precision", ctypes.c_int),
                ("local_bytes", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("setup_flops", ctypes.c_double),
                ("sweep_block", ctypes.c_int), ("tile_order", ctypes.c_int),
                ("ms_setup_tuned", ctypes.c_float), ("ms_setup_default", ctypes.c_float)]


class _GmresOptions(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_iters", ctypes.c_int), ("rtol", ctypes.c_double)]


class _GmresReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("rel_residual", ctypes.c_double)]


class _SolveOptions(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int), ("primal", ctypes.c_int), ("load_steps", ctypes.c_int),
        ("max_newton", ctypes.c_int), ("max_halvings", ctypes.c_int), ("restart", ctypes.c_int),
        ("max_gmres", ctypes.c_int), ("newton_rtol", ctypes.c_double), ("gmres_rtol", ctypes.c_double),
        ("pivot_tol", ctypes.c_double), ("levels", ctypes.c_int), ("n_parts2", ctypes.c_int),
        ("part2", _i32p), ("primal2", ctypes.c_int), ("precision2", ctypes.c_int),
        ("scaling", ctypes.c_int), ("coarse", ctypes.c_int), ("sweep_block", ctypes.c_int),
        ("tile_order", ctypes.c_int), ("autotune", ctypes.c_int),
    ]


class _Record(ctypes.Structure):
    _fields_ = [
        ("load", ctypes.c_double), ("newton", ctypes.c_int), ("gmres_its", ctypes.c_int),
        ("res", ctypes.c_double), ("res0", ctypes.c_double), ("ms_assemble", ctypes.c_float),
        ("ms_setup", ctypes.c_float), ("ms_gmres", ctypes.c_float), ("ms_total", ctypes.c_float),
        ("gmres_relres", ctypes.c_double), ("gmres_reorth", ctypes.c_int), ("ms_autotune", ctypes.c_float),
    ]


class _Report(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("newton_steps", ctypes.c_int), ("load_steps_done", ctypes.c_int),
        ("halvings", ctypes.c_int), ("total_gmres_its", ctypes.c_int),
        ("final_rel_residual", ctypes.c_double), ("n_records", ctypes.c_int),
        ("rec", _Record * MAX_RECORDS),
    ]


_LIB = None


def build(force=False):
    """Compile the CUDA library (sm_103a) in-tree; returns its path."""
    return _build.build(force=force)


def load_library():
    """Load libcardiac_bddc.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.lib_path()
    if not os.path.exists(path):
        raise ImportError("libcardiac_bddc.so is not built; call paper_2208_06191_gb300.build()")
    lib = ctypes.CDLL(path)
    vp, c_int, c_double = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "fem_problem_create": (c_int, [ctypes.POINTER(_Desc), ctypes.POINTER(vp)]),
        "fem_problem_destroy": (None, [vp]),
        "fem_problem_get_info": (c_int, [vp, ctypes.POINTER(_ProblemInfo)]),
        "fem_residual": (c_int, [vp, vp, c_double, vp, vp]),
        "fem_assemble_tangent": (c_int, [vp, vp, c_double, vp, ctypes.POINTER(_Tangent), vp]),
        "fem_spmv": (c_int, [vp, vp, vp, vp]),
        "fem_set_time_state": (c_int, [vp, c_double, vp, vp]),
        "fem_tangent_copy": (c_int, [vp, vp, vp, vp, vp]),
        "bddc_setup": (c_int, [vp, ctypes.POINTER(_Tangent), ctypes.POINTER(_BddcOptions),
                               ctypes.POINTER(vp), vp]),
        "bddc_apply": (c_int, [vp, vp, vp, vp]),
        "bddc_apply_noalloc": (c_int, [vp, vp, vp, vp]),
        "bddc_destroy": (None, [vp]),
        "bddc_get_info": (c_int, [vp, ctypes.POINTER(_BddcInfo)]),
        "gmres_solve": (c_int, [vp, vp, vp, vp, ctypes.POINTER(_GmresOptions),
                                ctypes.POINTER(_GmresReport), vp]),
        "newton_step": (c_int, [vp, ctypes.POINTER(vp), ctypes.POINTER(_SolveOptions), c_double, vp,
                                ctypes.POINTER(_Record), vp]),
        "newton_step_host": (c_int, [vp, ctypes.POINTER(vp), ctypes.POINTER(_SolveOptions), c_double, vp,
                                     ctypes.POINTER(_Record), vp]),
        "newton_gmres_solve": (c_int, [vp, ctypes.POINTER(_SolveOptions), vp, ctypes.POINTER(_Report), vp]),
        "cbddc_last_error": (ctypes.c_char_p, []),
        "cbddc_kernel_launches": (ctypes.c_uint64, []),
        "cbddc_set_tensor_cores": (c_int, [c_int]),
        "cbddc_timer_enable": (c_int, [c_int]),
        "cbddc_timer_result": (c_int, [c_int, ctypes.POINTER(c_double), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
        "cbddc_timer_start": (c_int, [c_int]),
        "cbddc_timer_stop": (c_int, [ctypes.POINTER(c_double), ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(c_double), ctypes.POINTER(c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def set_tensor_cores(mode):
    """FP32 setup GEMMs: mode bit 0 = tcgen05 tensor cores (else the FP32
    CUDA cores), bit 1 = three TF32 parts for the sweep updates, bit 2 =
    three parts for the other products, bits 3/4 = the other products / the
    sweep updates on the CUDA cores, bit 5 = sweep updates with a 32-wide K
    block per tensor-memory slice instead of one K-step, bit 6 = the other
    products with one K-step per slice instead of a 32-wide block
    (True means the default, 1; False means 0).  Returns the previous
    mode."""
    if mode is True:
        mode = 1
    elif mode is False:
        mode = 0
    return int(load_library().cbddc_set_tensor_cores(int(mode)))


def kernel_launches():
    """Kernels launched by the library since it was loaded."""
    return int(load_library().cbddc_kernel_launches())


def timer_start(kernel_class):
    """Record CUDA events around every launch of one kernel class."""
    _check(load_library().cbddc_timer_start(int(kernel_class)))


def timer_stop():
    """Returns dict(ms, launches, flops, bytes) of the recorded launches."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    fl, by = ctypes.c_double(), ctypes.c_double()
    _check(load_library().cbddc_timer_stop(ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fl),
                                           ctypes.byref(by)))
    return {"ms": ms.value, "launches": n.value, "flops": fl.value, "bytes": by.value}


def timer_enable(kernel_class):
    """Also record the launches of another kernel class."""
    _check(load_library().cbddc_timer_enable(int(kernel_class)))


def timer_result(kernel_class):
    """dict(ms, launches, flops, bytes) of one recorded class so far."""
    ms, n = ctypes.c_double(), ctypes.c_int64()
    fl, by = ctypes.c_double(), ctypes.c_double()
    _check(load_library().cbddc_timer_result(int(kernel_class), ctypes.byref(ms), ctypes.byref(n),
                                             ctypes.byref(fl), ctypes.byref(by)))
    return {"ms": ms.value, "launches": n.value, "flops": fl.value, "bytes": by.value}


def _check(rc):
    if rc != OK:
        raise CBDDCError(rc, _LIB.cbddc_last_error().decode())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError("expected dtype %s, got %s" % (dtype, t.dtype))
    return ctypes.c_void_p(t.data_ptr())


def _part2_arg(part2):
    if part2 is None:
        return None, None
    arr = np.ascontiguousarray(np.asarray(part2, dtype=np.int32))
    return arr, arr.ctypes.data_as(_i32p)


class SolveOptions:
    """Options of the Newton-GMRES-BDDC solve (see solve_options in the header).
    Multilevel BDDC: levels=3 with part2 (level-2 subdomain of every
    subdomain), n_parts2, primal2 and precision2 (level-2 local operators).
    scaling: "counting" or "deluxe" (first level); coarse: "galerkin" or
    "petrov" (left coarse basis from the transposed local problems);
    sweep_block: pivot block width of the local sweeps (0/64, or 128 for
    FP32 operators); tile_order: 1 orders the setup GEMM tiles largest
    problem first; autotune: time the candidates at context creation and
    keep the fastest."""

    def __init__(self, precision=FP64, primal="V", load_steps=4, max_newton=25, max_halvings=6,
                 restart=100, max_gmres=1000, newton_rtol=1e-8, gmres_rtol=1e-8, pivot_tol=1e-13,
                 levels=2, part2=None, n_parts2=0, primal2="VEF", precision2=FP64, scaling="counting",
                 coarse="galerkin", sweep_block=0, tile_order=0,
                 autotune=False):
        self.precision = precision
        self.primal = primal if isinstance(primal, int) else primal_mask(primal)
        self.load_steps = load_steps
        self.max_newton = max_newton
        self.max_halvings = max_halvings
        self.restart = restart
        self.max_gmres = max_gmres
        self.newton_rtol = newton_rtol
        self.gmres_rtol = gmres_rtol
        self.pivot_tol = pivot_tol
        self.levels = levels
        self.part2_arr, self._part2_ptr = _part2_arg(part2)
        self.n_parts2 = int(n_parts2)
        self.primal2 = primal2 if isinstance(primal2, int) else primal_mask(primal2)
        self.precision2 = precision2
        self.scaling = scaling_code(scaling)
        self.coarse = coarse_code(coarse)
        self.sweep_block = int(sweep_block)
        self.tile_order = int(tile_order)
        self.autotune = int(bool(autotune))

    def c(self):
        return _SolveOptions(self.precision, self.primal, self.load_steps, self.max_newton,
                             self.max_halvings, self.restart, self.max_gmres, self.newton_rtol,
                             self.gmres_rtol, self.pivot_tol, self.levels, self.n_parts2,
                             self._part2_ptr, self.primal2, self.precision2, self.scaling, self.coarse,
                             self.sweep_block, self.tile_order, self.autotune)


def _record_dict(r):
    return {k: getattr(r, k) for k, _ in _Record._fields_}


class Problem:
    """A discretised problem on the current CUDA device (fem_problem).

    ``prob`` is a dict (the generators in ``workloads`` build them):

    * ``elem_type``: "Q1", "Q2" (hexahedra; local node a + (k+1)(b +
      (k+1)c) at reference position (a, b, c)/k) or "P1", "P2" (tetrahedra:
      4 corners, then the mid-nodes of edges 01, 12, 02, 03, 13, 23);
    * ``coords`` (n_nodes, 3) reference coordinates; ``elems`` (n_el, n_en)
      node ids; ``elem_part`` (n_el,) subdomain of every element and
      ``n_parts``;
    * ``dirichlet_nodes``: clamped nodes (all three components);
    * ``pressure_faces`` (n, 2): (element, local face) pairs carrying the
      follower pressure ``pressure`` (Pa, scaled by the load factor);
    * ``fibers``: {"kind": "slab_helix", "z0", "z1", "alpha0", "alpha1"}
      (angle rising linearly in z, degrees) or {"kind": "nodal", "f", "n"}
      (fibre and sheet-normal directions per node, (n_nodes, 3) each);
    * ``material``: Guccione constants C, bff, bss, bnn, bfs, bfn, bsn and
      the bulk modulus B (Pa); ``gamma``: active tension (Pa, scaled by the
      load factor);
    * optional, for the time-dependent model: ``rho`` (density),
      ``robin_faces`` (n, 3) rows (element, local face, parameter set 0/1)
      and ``robin``, two dicts with k_perp, k_par, c_perp, c_par.
    """

    def __init__(self, prob):
        lib = load_library()
        self._keep = []

        def i32(a):
            a = np.ascontiguousarray(np.asarray(a, dtype=np.int32))
            self._keep.append(a)
            return a.ctypes.data_as(_i32p)

        coords = np.ascontiguousarray(np.asarray(prob["coords"], dtype=np.float64))
        self._keep.append(coords)
        et = {"Q1": HEX_Q1, "Q2": HEX_Q2, "P1": TET_P1, "P2": TET_P2}[prob["elem_type"]]
        fib = prob["fibers"]
        if fib["kind"] not in ("slab_helix", "nodal"):
            raise ValueError("unsupported fibre field %r" % fib["kind"])
        mat = prob["material"]
        d = _Desc()
        d.elem_type = et
        d.n_nodes = coords.shape[0]
        d.coords = coords.ctypes.data_as(_dp)
        d.n_elems = len(prob["elems"])
        d.elems = i32(prob["elems"])
        d.elem_part = i32(prob["elem_part"])
        d.n_parts = int(prob["n_parts"])
        d.n_dirichlet = len(prob["dirichlet_nodes"])
        d.dirichlet_nodes = i32(prob["dirichlet_nodes"])
        pf = np.asarray(prob["pressure_faces"], dtype=np.int32).reshape(-1, 2)
        d.n_pressure_faces = pf.shape[0]
        d.pressure_faces = i32(pf)
        if fib["kind"] == "slab_helix":
            d.fiber_kind = FIBER_SLAB_HELIX
            for i, v in enumerate([fib["z0"], fib["z1"], fib["alpha0"], fib["alpha1"]]):
                d.fiber_params[i] = float(v)
        else:
            d.fiber_kind = FIBER_NODAL
            fn = np.ascontiguousarray(np.hstack([np.asarray(fib["f"], dtype=np.float64),
                                                 np.asarray(fib["n"], dtype=np.float64)]))
            if fn.shape != (coords.shape[0], 6):
                raise ValueError("nodal fibres must have one (f, n) pair per node")
            self._keep.append(fn)
            d.fiber_nodal = fn.ctypes.data_as(_dp)
        for i, k in enumerate(["C", "bff", "bss", "bnn", "bfs", "bfn", "bsn", "B"]):
            d.material[i] = float(mat[k])
        d.pressure = float(prob["pressure"])
        d.gamma = float(prob["gamma"])
        # time-dependent terms: density and Robin faces (optional keys)
        d.rho = float(prob.get("rho", 0.0))
        rf = np.asarray(prob.get("robin_faces", np.zeros((0, 3))), dtype=np.int32).reshape(-1, 3)
        d.n_robin_faces = rf.shape[0]
        d.robin_faces = i32(rf)
        for q, par in enumerate(prob.get("robin", [])[:2]):
            for c, key in enumerate(("k_perp", "k_par", "c_perp", "c_par")):
                d.robin[q][c] = float(par[key])
        h = ctypes.c_void_p()
        _check(lib.fem_problem_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self._keep = []
        self.prob = prob
        self.info = self._info()
        self.n_free = int(self.info["n_free"])

    def _info(self):
        inf = _ProblemInfo()
        _check(_LIB.fem_problem_get_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in _ProblemInfo._fields_}

    def close(self):
        if getattr(self, "_h", None):
            _LIB.fem_problem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def residual(self, d, load, out):
        import torch
        _check(_LIB.fem_residual(self._h, _ptr(d, torch.float64), float(load),
                                 _ptr(out, torch.float64), _stream()))
        return out

    def assemble_tangent(self, d, load, residual=None):
        """Residual (into ``residual`` if given) and tangent; returns a dict
        viewing the device BSR arrays (valid until the next assembly)."""
        import torch
        K = _Tangent()
        rp = _ptr(residual, torch.float64) if residual is not None else None
        _check(_LIB.fem_assemble_tangent(self._h, _ptr(d, torch.float64), float(load), rp,
                                         ctypes.byref(K), _stream()))
        self._tangent = K
        return {"vals": K.vals, "row_ptr": K.row_ptr, "col_idx": K.col_idx,
                "n_block_rows": K.n_block_rows, "nnzb": K.nnzb}

    def spmv(self, x, y):
        import torch
        _check(_LIB.fem_spmv(self._h, _ptr(x, torch.float64), _ptr(y, torch.float64), _stream()))
        return y

    def set_time_state(self, dt, d_prev=None, d_prev2=None):
        """Backward-Euler step dt with the two previous displacements (CUDA
        FP64 tensors, kept referenced here while the state is set); dt = 0
        returns to the quasi-static problem."""
        import torch
        if dt and dt > 0:
            self._time_keep = (d_prev, d_prev2)
            _check(_LIB.fem_set_time_state(self._h, float(dt), _ptr(d_prev, torch.float64),
                                           _ptr(d_prev2, torch.float64)))
        else:
            _check(_LIB.fem_set_time_state(self._h, 0.0, None, None))
            self._time_keep = None

    def tangent_to_host(self):
        """Copies the last tangent to host numpy arrays:
        (vals [nnzb,3,3], row_ptr [n+1], col_idx [nnzb])."""
        import torch
        K = self._tangent
        vals = torch.empty(K.nnzb * 9, dtype=torch.float64, device="cuda")
        rp = torch.empty(K.n_block_rows + 1, dtype=torch.int32, device="cuda")
        ci = torch.empty(K.nnzb, dtype=torch.int32, device="cuda")
        _check(_LIB.fem_tangent_copy(self._h, _ptr(vals), _ptr(rp), _ptr(ci), _stream()))
        return (vals.cpu().numpy().reshape(-1, 3, 3), rp.cpu().numpy(), ci.cpu().numpy())

    def newton_step(self, d, load, options, ctx=None, host=False):
        """One Newton step (assemble, BDDC setup, GMRES, update d in place).
        ``d``: CUDA FP64 tensor, or a host FP64 numpy array with host=True.
        Returns (record dict, BDDC context)."""
        import torch
        rec = _Record()
        h = ctypes.c_void_p(ctx._h.value if ctx is not None else None)
        opt = options.c()
        if host:
            arr = d
            assert isinstance(arr, np.ndarray) and arr.dtype == np.float64 and arr.flags.c_contiguous
            rc = _LIB.newton_step_host(self._h, ctypes.byref(h), ctypes.byref(opt), float(load),
                                       ctypes.c_void_p(arr.ctypes.data), ctypes.byref(rec), _stream())
        else:
            rc = _LIB.newton_step(self._h, ctypes.byref(h), ctypes.byref(opt), float(load),
                                  _ptr(d, torch.float64), ctypes.byref(rec), _stream())
        if ctx is None and h.value:
            ctx = BDDC._wrap(h, self)
        if rc not in (OK, ENOCONV):
            _check(rc)
        out = _record_dict(rec)
        out["status"] = rc
        return out, ctx

    def solve(self, options, d=None):
        """Full load-stepped Newton solve; returns (d, report dict)."""
        import torch
        if d is None:
            d = torch.zeros(self.n_free, dtype=torch.float64, device="cuda")
        rep = _Report()
        rc = _LIB.newton_gmres_solve(self._h, ctypes.byref(options.c()), _ptr(d, torch.float64),
                                     ctypes.byref(rep), _stream())
        _check(rc)
        out = {k: getattr(rep, k) for k, _ in _Report._fields_ if k != "rec"}
        out["records"] = [_record_dict(rep.rec[i]) for i in range(rep.n_records)]
        return d, out


class BDDC:
    """BDDC preconditioner context (bddc_ctx) for a problem."""

    def __init__(self, problem, precision=FP64, primal="V", pivot_tol=1e-13, levels=2, part2=None,
                 n_parts2=0, primal2="VEF", precision2=FP64, scaling="counting", coarse="galerkin",
                 sweep_block=0, tile_order=0):
        self.problem = problem
        self._h = ctypes.c_void_p()
        self._part2, p2 = _part2_arg(part2)
        self._opt = _BddcOptions(precision, primal if isinstance(primal, int) else primal_mask(primal),
                                 pivot_tol, levels, int(n_parts2), p2,
                                 primal2 if isinstance(primal2, int) else primal_mask(primal2),
                                 precision2, scaling_code(scaling), coarse_code(coarse), int(sweep_block),
                                 int(tile_order))

    @classmethod
    def _wrap(cls, h, problem):
        obj = cls.__new__(cls)
        obj.problem = problem
        obj._h = h
        obj._opt = None
        return obj

    def setup(self):
        K = getattr(self.problem, "_tangent", None)
        _check(_LIB.bddc_setup(self.problem.handle, ctypes.byref(K) if K is not None else None,
                               ctypes.byref(self._opt), ctypes.byref(self._h), _stream()))
        return self

    def apply(self, r, z):
        import torch
        _check(_LIB.bddc_apply(self._h, _ptr(r, torch.float64), _ptr(z, torch.float64), _stream()))
        return z

    def apply_noalloc(self, r, z):
        """z = M^-1 r with the work vectors in the library's static device
        array (no device allocation during the call)."""
        import torch
        _check(_LIB.bddc_apply_noalloc(self._h, _ptr(r, torch.float64), _ptr(z, torch.float64),
                                       _stream()))
        return z

    def info(self):
        inf = _BddcInfo()
        _check(_LIB.bddc_get_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in _BddcInfo._fields_}

    def gmres(self, b, x, restart=100, max_iters=1000, rtol=1e-8):
        import torch
        rep = _GmresReport()
        opt = _GmresOptions(restart, max_iters, rtol)
        rc = _LIB.gmres_solve(self.problem.handle, self._h, _ptr(b, torch.float64),
                              _ptr(x, torch.float64), ctypes.byref(opt), ctypes.byref(rep), _stream())
        if rc not in (OK, ENOCONV):
            _check(rc)
        return {"iterations": rep.iterations, "converged": bool(rep.converged),
                "rel_residual": rep.rel_residual, "status": rc}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _LIB.bddc_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
