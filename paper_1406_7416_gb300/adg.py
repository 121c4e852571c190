"""Thin ctypes binding of libadg (include/adg.h): argument marshalling only.

Every step of the time step runs in the library's CUDA kernels; this module
converts numpy arrays and Python scalars into the C ABI's pointers and sizes.
It raises when libadg.so is missing -- there is no fallback path.

Host array layouts follow include/adg.h: dofs[cell][var][node],
sub[cell][var][subcell], beta[cell], with x fastest in every index.
"""
import ctypes
import os

import numpy as np

from . import inputs

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libadg.so")

OK = 0
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_CAPACITY, ERR_STATE = -1, -2, -3, -4, -5, -6
WARN_SUBCELL_INADMISSIBLE = 1
BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE, BC_INFLOW, BC_FRONT = 0, 1, 2, 3, 4
PREC_FP64, PREC_MIXED_FP32, PREC_MIXED_TF32 = 0, 1, 2
OPT_DMP_EPS, OPT_DMP_FLOOR, OPT_FORCE_LIMITER, OPT_PICARD_ITERS, OPT_SLOT_CAPACITY = 1, 2, 3, 4, 5
OPT_PROFILE = 6
OPT_FP64_SWEEPS = 7
OPT_END_TIME = 8
OPT_CFL = 9
OPT_SCRATCH_BYTES = 10
OPT_CASCADE = 11
OPT_FLUX = 12
OPT_HOST_PASSES = 13
OPT_SUBCELL_FP64_SWEEPS = 14
OPT_SUBCELL_FP32 = 15
OPT_PROJECT_DELTA = 16
OPT_PREDICTOR = 17
OPT_SUBCELL_REGISTERS = 18
PRED_BLOCK, PRED_BLOCK_ALT, PRED_WARP2, PRED_WARP4, PRED_WARP4_TC, PRED_WARP1 = 0, 1, 2, 3, 4, 5
PRED_NAMES = ("block", "block_alt", "warp2", "warp4", "warp4_tc", "warp1")
FLUX_RUSANOV, FLUX_OSHER = 0, 1
PHASES = ("predictor", "faceflux", "correct_detect", "limiter", "fix")
IC_RADIAL, IC_QUADRANT, IC_PLANAR = 0, 1, 2

# every entry point declared in include/adg.h
SYMBOLS = ("adg_create", "adg_set_allocator", "adg_set_stream", "adg_set_option", "adg_load",
           "adg_init_problem", "adg_load_full", "adg_read_full", "adg_step", "adg_step_cfl",
           "adg_max_dt", "adg_flags", "adg_read", "adg_troubled_count", "adg_status",
           "adg_sizes", "adg_info", "adg_phase_times", "adg_last_error", "adg_destroy",
           "adg_subcell_update_noalloc", "adg_time", "adg_batch_create", "adg_batch_step",
           "adg_batch_destroy", "adg_step_batch", "adg_fallback_count", "adg_set_boundary_state",
           "adg_set_boundary_front", "adg_set_time", "adg_autotune", "adg_troubled_history",
           "adg_halo_bytes", "adg_pack_cells", "adg_unpack_cells", "adg_pipe_rates")


class AdgGrid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("x0", ctypes.c_double * 3),
                ("dx", ctypes.c_double * 3)]


class AdgProblem(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("center", ctypes.c_double * 3),
                ("radius", ctypes.c_double), ("inner", ctypes.c_double * 5),
                ("outer", ctypes.c_double * 5), ("quad", (ctypes.c_double * 4) * 4),
                ("vortex", ctypes.c_int), ("vortex_center", ctypes.c_double * 2),
                ("vortex_strength", ctypes.c_double),
                ("cell_rho_factor", ctypes.POINTER(ctypes.c_double)),
                ("normal", ctypes.c_double * 3), ("offset", ctypes.c_double)]


class AdgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libadg error {code}: {msg}")
        self.code = code


_lib = None


def load_library(path=None):
    """Load libadg.so (built in-tree by build_lib.py); raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libadg.so not found at {p}: run paper_1406_7416_gb300.build_lib.build()")
    lib = ctypes.CDLL(p)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    lib.adg_create.argtypes = [ctypes.POINTER(AdgGrid), ip, ctypes.c_double,
                               ctypes.POINTER(ctypes.c_int), ip, ctypes.POINTER(vp)]
    lib.adg_set_allocator.argtypes = [vp, vp, vp, vp]
    lib.adg_set_stream.argtypes = [vp, vp]
    lib.adg_set_option.argtypes = [vp, ip, ctypes.c_double]
    lib.adg_load.argtypes = [vp, dp, dp]
    lib.adg_init_problem.argtypes = [vp, ctypes.POINTER(AdgProblem)]
    lib.adg_load_full.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_uint8), dp]
    lib.adg_read_full.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_uint8), dp]
    lib.adg_step.argtypes = [vp, ctypes.c_double]
    lib.adg_step_cfl.argtypes = [vp, ctypes.c_double, ctypes.c_double]
    lib.adg_max_dt.argtypes = [vp, ctypes.c_double, dp]
    lib.adg_flags.argtypes = [vp, ctypes.POINTER(ctypes.c_uint8)]
    lib.adg_read.argtypes = [vp, dp]
    lib.adg_troubled_count.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    lib.adg_fallback_count.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.adg_set_boundary_state.argtypes = [vp, ip, dp]
    lib.adg_set_boundary_front.argtypes = [vp, ip, ip, ctypes.c_double, ctypes.c_double, ip, dp, ip, dp]
    lib.adg_set_time.argtypes = [vp, ctypes.c_double]
    lib.adg_status.argtypes = [vp]
    lib.adg_sizes.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.adg_phase_times.argtypes = [vp, dp, ip]
    lib.adg_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ip]
    lib.adg_autotune.argtypes = [vp, ip, dp, ip]
    lib.adg_pipe_rates.argtypes = [dp, ip]
    ipp = ctypes.POINTER(ctypes.c_int)
    lib.adg_halo_bytes.argtypes = [vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    lib.adg_pack_cells.argtypes = [vp, ipp, ipp, vp]
    lib.adg_unpack_cells.argtypes = [vp, ipp, ipp, vp]
    lib.adg_troubled_history.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ip,
                                         ctypes.POINTER(ctypes.c_int)]
    lib.adg_last_error.argtypes = [vp]
    lib.adg_last_error.restype = ctypes.c_char_p
    lib.adg_subcell_update_noalloc.argtypes = [ip, ip, ctypes.c_double, dp, ctypes.c_double, vp, ip,
                                               vp, vp, vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.adg_destroy.argtypes = [vp]
    lib.adg_destroy.restype = None
    lib.adg_time.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_int64)]
    lib.adg_batch_create.argtypes = [ctypes.POINTER(vp), ip, vp, ctypes.POINTER(vp)]
    lib.adg_batch_step.argtypes = [vp, dp, ctypes.c_double]
    lib.adg_batch_destroy.argtypes = [vp]
    lib.adg_batch_destroy.restype = None
    lib.adg_step_batch.argtypes = [ctypes.POINTER(vp), dp, ip]
    for name in SYMBOLS:
        if name not in ("adg_last_error", "adg_destroy", "adg_batch_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _contig(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def pipe_rates():
    """adg_pipe_rates: {pipe: thread operations per second} of the current device, and the
    Newton reciprocal's largest difference from 1.0 / x (ulps) with the fraction that differs."""
    lib = load_library()
    out = np.zeros(8)
    rc = lib.adg_pipe_rates(_dptr(out), 8)
    if rc != OK:
        raise AdgError(rc, "adg_pipe_rates failed")
    return dict(zip(("dfma", "ffma", "f64_to_f32", "f64_compare", "f64_reciprocal_div",
                     "f64_reciprocal_newton", "newton_max_ulp", "newton_differ_fraction"),
                    out.tolist()))


def subcell_update_noalloc(dim, N, gamma, h, dt, patches_ptr, count, vnew_ptr, faces_ptr=0,
                           stream=0):
    """adg_subcell_update_noalloc on caller-owned device buffers (raw pointers).
    Returns the status code and the library's message."""
    lib = load_library()
    hh = np.ascontiguousarray(h, dtype=np.float64)
    err = ctypes.create_string_buffer(512)
    rc = lib.adg_subcell_update_noalloc(int(dim), int(N), float(gamma), _dptr(hh), float(dt),
                                        ctypes.c_void_p(int(patches_ptr)), int(count),
                                        ctypes.c_void_p(int(vnew_ptr)),
                                        ctypes.c_void_p(int(faces_ptr)) if faces_ptr else None,
                                        ctypes.c_void_p(int(stream)) if stream else None,
                                        err, 512)
    return rc, err.value.decode()


class Solver:
    """One libadg state: grid, degree, gamma, boundary kinds, precision."""

    def __init__(self, dim, ncell, x0, dx, bc, N, gamma=1.4, prec=PREC_FP64):
        self.lib = load_library()
        g = AdgGrid()
        g.dim = dim
        for k in range(3):
            g.n[k] = int(ncell[k]) if k < dim else 1
            g.x0[k] = float(x0[k]) if k < dim else 0.0
            g.dx[k] = float(dx[k]) if k < dim else 1.0
        bcs = (ctypes.c_int * 6)(*([int(b) for b in bc] + [0] * (6 - len(bc))))
        h = ctypes.c_void_p()
        rc = self.lib.adg_create(ctypes.byref(g), int(N), float(gamma), bcs, int(prec), ctypes.byref(h))
        if rc != OK:
            raise AdgError(rc, "adg_create rejected its arguments")
        self.h = h
        self.dim, self.N, self.gamma, self.prec = dim, N, gamma, prec
        self.ncell = tuple(int(c) for c in ncell[:dim])
        c, nv, nd, ns = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self.lib.adg_sizes(h, ctypes.byref(c), ctypes.byref(nv), ctypes.byref(nd), ctypes.byref(ns))
        self.cells, self.nvar, self.nodes, self.subcells = c.value, nv.value, nd.value, ns.value
        self._keep = []

    @classmethod
    def from_workload(cls, w, prec=PREC_FP64):
        s = cls(w["dim"], w["ncell"], w["x0"], w["dx"], w["bc"], w["N"], w["gamma"], prec)
        for face, q in (w.get("bc_states") or {}).items():
            s.set_boundary_state(face, q)
        for face, fr in (w.get("bc_fronts") or {}).items():
            s.set_boundary_front(face, fr["axis"], fr["a"], fr["b"], fr["before"], fr["after"])
        return s

    def set_boundary_front(self, face, axis, a, b, before, after):
        """Moving split of front face `face`; before / after = (kind, state or None)."""
        def arg(q):
            if q is None:
                return None, None
            arr = np.ascontiguousarray(q, dtype=np.float64)
            return arr, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        qb, pb = arg(before[1])
        qa, pa = arg(after[1])
        self._check(self.lib.adg_set_boundary_front(self.h, int(face), int(axis), float(a), float(b),
                                                    int(before[0]), pb, int(after[0]), pa),
                    "adg_set_boundary_front")

    def set_time(self, t):
        """Set the simulated time (restarts, time-dependent boundaries)."""
        self._check(self.lib.adg_set_time(self.h, float(t)), "adg_set_time")

    def set_boundary_state(self, face, q):
        """Conserved state of inflow face `face` (2k low, 2k+1 high of axis k)."""
        a = np.ascontiguousarray(q, dtype=np.float64)
        self._check(self.lib.adg_set_boundary_state(self.h, int(face),
                                                     a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                    "adg_set_boundary_state")

    # -- helpers ------------------------------------------------------------
    def _check(self, rc, what):
        if rc < 0:
            raise AdgError(rc, f"{what}: {self.lib.adg_last_error(self.h).decode()}")
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.adg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- configuration ------------------------------------------------------
    def set_option(self, key, value):
        self._check(self.lib.adg_set_option(self.h, int(key), float(value)), "adg_set_option")

    def set_stream(self, stream_handle):
        self._check(self.lib.adg_set_stream(self.h, ctypes.c_void_p(int(stream_handle))),
                    "adg_set_stream")

    def use_torch_allocator(self):
        """Route the state's device allocations through torch's caching allocator."""
        import torch
        AllocT = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
        FreeT = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
        dev = torch.cuda.current_device()

        def _alloc(nbytes, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev)
            except RuntimeError:
                return None

        def _free(ptr, ctx):
            torch.cuda.caching_allocator_delete(int(ptr))

        a, f = AllocT(_alloc), FreeT(_free)
        self._keep += [a, f]
        self._check(self.lib.adg_set_allocator(self.h, ctypes.cast(a, ctypes.c_void_p),
                                               ctypes.cast(f, ctypes.c_void_p), None),
                    "adg_set_allocator")

    # -- data in / out ------------------------------------------------------
    def load(self, dofs, exact=None):
        d = _contig(dofs, np.float64)
        assert d.size == self.cells * self.nvar * self.nodes
        e = None if exact is None else _contig(exact, np.float64)
        self._check(self.lib.adg_load(self.h, _dptr(d), None if e is None else _dptr(e)),
                    "adg_load")

    def init_problem(self, problem):
        pr = AdgProblem()
        fac = None
        if problem["kind"] == "radial":
            pr.kind = IC_RADIAL
            for k, c in enumerate(problem["center"]):
                pr.center[k] = c
            pr.radius = problem["radius"]
            for k, v in enumerate(problem["inner"]):
                pr.inner[k] = v
            for k, v in enumerate(problem["outer"]):
                pr.outer[k] = v
            if problem.get("cell_rho_factor") is not None:
                # per-cell factors in the ABI's cell order (x fastest)
                fac = _contig(np.asarray(problem["cell_rho_factor"]).transpose().ravel(), np.float64)
                pr.cell_rho_factor = _dptr(fac)
        elif problem["kind"] == "planar":
            pr.kind = IC_PLANAR
            for k, c in enumerate(problem["normal"]):
                pr.normal[k] = c
            pr.offset = problem["offset"]
            for k, v in enumerate(problem["inner"]):
                pr.inner[k] = v
            for k, v in enumerate(problem["outer"]):
                pr.outer[k] = v
        else:
            pr.kind = IC_QUADRANT
            pr.center[0], pr.center[1] = problem["center"]
            for q in range(4):
                for k in range(4):
                    pr.quad[q][k] = problem["states"][q][k]
            vx = problem.get("vortex")
            if vx is not None:
                pr.vortex = 1
                pr.vortex_center[0], pr.vortex_center[1] = vx["center"]
                pr.vortex_strength = vx["strength"]
        self._check(self.lib.adg_init_problem(self.h, ctypes.byref(pr)), "adg_init_problem")

    def load_full(self, dofs, beta, sub):
        d = _contig(dofs, np.float64)
        b = _contig(beta, np.uint8)
        s = _contig(sub, np.float64)
        self._check(self.lib.adg_load_full(self.h, _dptr(d), _u8ptr(b), _dptr(s)), "adg_load_full")

    def read(self, out=None):
        out = np.empty((self.cells, self.nvar, self.nodes)) if out is None else out
        self._check(self.lib.adg_read(self.h, _dptr(out)), "adg_read")
        return out

    def read_full(self):
        d = np.empty((self.cells, self.nvar, self.nodes))
        b = np.empty(self.cells, dtype=np.uint8)
        s = np.empty((self.cells, self.nvar, self.subcells))
        self._check(self.lib.adg_read_full(self.h, _dptr(d), _u8ptr(b), _dptr(s)), "adg_read_full")
        return d, b, s

    def flags(self):
        b = np.empty(self.cells, dtype=np.uint8)
        self._check(self.lib.adg_flags(self.h, _u8ptr(b)), "adg_flags")
        return b

    def troubled_count(self):
        c = ctypes.c_int64()
        self._check(self.lib.adg_troubled_count(self.h, ctypes.byref(c)), "adg_troubled_count")
        return c.value

    # -- halo exchange of a domain decomposition ----------------------------
    def halo_bytes(self, count):
        b = ctypes.c_int64()
        self._check(self.lib.adg_halo_bytes(self.h, int(count), ctypes.byref(b)), "adg_halo_bytes")
        return b.value

    @staticmethod
    def _box(lo, hi):
        return (ctypes.c_int * 3)(*(list(lo) + [0] * (3 - len(lo)))), \
               (ctypes.c_int * 3)(*(list(hi) + [1] * (3 - len(hi))))

    def pack_cells(self, lo, hi, buf_ptr):
        """adg_pack_cells into the device buffer at buf_ptr (raw pointer)."""
        a, b = self._box(lo, hi)
        self._check(self.lib.adg_pack_cells(self.h, a, b, ctypes.c_void_p(int(buf_ptr))),
                    "adg_pack_cells")

    def unpack_cells(self, lo, hi, buf_ptr):
        a, b = self._box(lo, hi)
        self._check(self.lib.adg_unpack_cells(self.h, a, b, ctypes.c_void_p(int(buf_ptr))),
                    "adg_unpack_cells")

    def troubled_history(self, max_steps=4096):
        """Troubled-cell counts of the last steps since the load, oldest first."""
        out = np.zeros(max_steps, dtype=np.int64)
        k = ctypes.c_int()
        self._check(self.lib.adg_troubled_history(
            self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(max_steps),
            ctypes.byref(k)), "adg_troubled_history")
        return out[:k.value]

    def fallback_count(self):
        """(cells recomputed by the first-order layer in the last step, since the load)."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._check(self.lib.adg_fallback_count(self.h, ctypes.byref(a), ctypes.byref(b)),
                    "adg_fallback_count")
        return a.value, b.value

    def status(self):
        return self._check(self.lib.adg_status(self.h), "adg_status")

    # -- time stepping ------------------------------------------------------
    def step(self, dt):
        self._check(self.lib.adg_step(self.h, float(dt)), "adg_step")

    def step_cfl(self, cfl, dt_max=-1.0):
        self._check(self.lib.adg_step_cfl(self.h, float(cfl), float(dt_max)), "adg_step_cfl")

    def phase_times(self):
        """{phase: accumulated ms} and the number of steps timed (profiling on)."""
        ms = np.zeros(8)
        self._check(self.lib.adg_phase_times(self.h, _dptr(ms), 8), "adg_phase_times")
        return dict(zip(PHASES, ms[:5].tolist())), int(ms[5])

    def info(self):
        """Slot capacity, limiter chunk, kernels of one adg_step at most, device
        bytes held, kernels issued by the steps so far, Picard sweeps, how
        many run in FP64, and the predictor's launch shape in effect."""
        out = (ctypes.c_int64 * 8)()
        self._check(self.lib.adg_info(self.h, out, 8), "adg_info")
        return dict(capacity=out[0], chunk=out[1], launches_per_step=out[2], bytes=out[3],
                    launches=out[4], picard_iters=out[5], fp64_sweeps=out[6],
                    predictor=int(out[7]))

    def autotune(self, reps=3):
        """adg_autotune: {shape name: ms per predictor launch} (NaN: n/a);
        the state keeps the fastest shape."""
        ms = np.zeros(len(PRED_NAMES))
        self._check(self.lib.adg_autotune(self.h, int(reps), _dptr(ms), len(ms)), "adg_autotune")
        return dict(zip(PRED_NAMES, ms.tolist()))

    def time(self):
        """(simulated time, steps taken since the last load)."""
        t, n = ctypes.c_double(), ctypes.c_int64()
        self._check(self.lib.adg_time(self.h, ctypes.byref(t), ctypes.byref(n)), "adg_time")
        return t.value, n.value

    def bytes_held(self):
        return self.info()["bytes"]

    def max_dt(self, cfl):
        dt = ctypes.c_double()
        self._check(self.lib.adg_max_dt(self.h, float(cfl), ctypes.byref(dt)), "adg_max_dt")
        return dt.value


def _handles(solvers):
    arr = (ctypes.c_void_p * len(solvers))()
    for i, s in enumerate(solvers):
        arr[i] = s.h
    return arr


class Batch:
    """adg_batch: states of equal (dim, N, precision) share every launch; CFL
    steps replay as one CUDA graph from the second step on."""

    def __init__(self, solvers, stream=0):
        self.lib = load_library()
        self.solvers = list(solvers)
        h = ctypes.c_void_p()
        rc = self.lib.adg_batch_create(_handles(self.solvers), len(self.solvers),
                                       ctypes.c_void_p(int(stream)) if stream else None,
                                       ctypes.byref(h))
        if rc != OK:
            raise AdgError(rc, "adg_batch_create failed")
        self.h = h

    def step(self, dts=None, cfl=0.0):
        if dts is not None:
            d = _contig(dts, np.float64)
            rc = self.lib.adg_batch_step(self.h, _dptr(d), 0.0)
        else:
            rc = self.lib.adg_batch_step(self.h, None, float(cfl))
        if rc < 0:
            msg = self.lib.adg_last_error(self.solvers[0].h).decode()
            raise AdgError(rc, f"adg_batch_step: {msg}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.adg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def step_batch(solvers, dts):
    """adg_step_batch: one step of every solver, shared launches."""
    lib = load_library()
    d = _contig(dts, np.float64)
    rc = lib.adg_step_batch(_handles(solvers), _dptr(d), len(solvers))
    if rc < 0:
        raise AdgError(rc, "adg_step_batch: " + lib.adg_last_error(solvers[0].h).decode())


__all__ = ["Solver", "Batch", "step_batch", "AdgError", "load_library", "SYMBOLS", "inputs"]
