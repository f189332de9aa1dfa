"""ctypes binding of libfsei.so (include/fsei.h): argument marshalling only.

Every step of the fractional-step integrator runs in the library's CUDA
kernels; torch tensors only supply device memory and the CUDA stream.  The
library is loaded on first use and a missing or unloadable library raises
``FseiUnavailable`` -- there is no fallback.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfsei.so")

FSEI_OK = 0
STATUS_NAMES = {0: "FSEI_OK", 1: "FSEI_E_ARG", 2: "FSEI_E_SHAPE",
                3: "FSEI_E_UNSUPPORTED", 4: "FSEI_E_NOMEM", 5: "FSEI_E_CUDA",
                6: "FSEI_E_NONFINITE", 7: "FSEI_E_CFL", 8: "FSEI_E_BOUNDS"}
FSEI_FP64, FSEI_MIXED = 0, 1
FSEI_Z_PERIODIC, FSEI_Z_WALLS = 0, 1
FSEI_AB2_CN, FSEI_RK3_CN = 0, 1
FSEI_NEWTONIAN, FSEI_CARREAU_YASUDA = 0, 1
FLAG_NONFINITE, FLAG_CFL = 1, 2

# exported symbols and their C signatures (kept in step with include/fsei.h)
EXPORTS = ("fsei_grid_create", "fsei_grid_destroy", "fsei_grid_workspace_bytes",
           "fsei_step", "fsei_step_host", "fsei_step_host_join", "fsei_poisson_solve", "fsei_adjoint_step", "fsei_batch_create",
           "fsei_batch_destroy", "fsei_batch_size", "fsei_batch_step", "fsei_set_kernel_timing",
           "fsei_kernel_times", "fsei_kernel_name", "fsei_last_error", "fsei_version",
           "fsei_grid_autotune", "fsei_grid_get_schedule", "fsei_grid_set_schedule",
           "fsei_batch_autotune", "fsei_fp64_fma_rate", "fsei_batch_set_max_group",
           "fsei_batch_launch_groups", "fsei_ib_forcing", "fsei_ib_loads",
           "fsei_grid_check_bounds", "fsei_grid_poke_guard")
FSEI_TUNE_FORCE = 1


class FseiUnavailable(RuntimeError):
    pass


class FseiError(RuntimeError):
    """A non-OK status.  stats: the statistics the call filled (a dict, or a
    list of dicts for a batch) when it reports a device flag, else None."""

    def __init__(self, status, message, stats=None):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status
        self.stats = stats


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double),
                ("zbc", ctypes.c_int32), ("lz", ctypes.c_double),
                ("stretch", ctypes.c_double),
                ("zfaces", ctypes.POINTER(ctypes.c_double)),
                ("prec", ctypes.c_int32), ("near_zero_tau", ctypes.c_double)]


class State(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("v", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("p", ctypes.c_void_p), ("hu", ctypes.c_void_p), ("hv", ctypes.c_void_p),
                ("hw", ctypes.c_void_p), ("have_prev_h", ctypes.c_int32)]


class CarreauYasuda(ctypes.Structure):
    _fields_ = [("lam", ctypes.c_double), ("n", ctypes.c_double), ("a", ctypes.c_double),
                ("eta_inf", ctypes.c_double)]


class StepParams(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("dt", ctypes.c_double), ("cfl", ctypes.c_double),
                ("gamma", ctypes.c_double), ("rho", ctypes.c_double),
                ("fconst", ctypes.c_double * 3), ("scheme", ctypes.c_int32),
                ("rheology", ctypes.c_int32), ("cy", CarreauYasuda)]


def _rheology(cy):
    """(rheology flag, CarreauYasuda) of None or a dict lam, n, a, eta_inf."""
    if cy is None:
        return FSEI_NEWTONIAN, CarreauYasuda(0.0, 1.0, 1.0, 1.0)
    return FSEI_CARREAU_YASUDA, CarreauYasuda(cy["lam"], cy["n"], cy["a"], cy["eta_inf"])


class StepStats(ctypes.Structure):
    _fields_ = [("dt_used", ctypes.c_double), ("cfl", ctypes.c_double),
                ("max_div", ctypes.c_double), ("kinetic_energy", ctypes.c_double),
                ("flags", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Schedule(ctypes.Structure):
    _fields_ = [("rhs_cells_per_lane", ctypes.c_int32),
                ("poisson_lanes_per_line", ctypes.c_int32),
                ("poisson_rows_per_lane", ctypes.c_int32),
                ("rfft_rows_per_block", ctypes.c_int32),
                ("ffty_columns_per_block", ctypes.c_int32),
                ("project_passes_per_thread", ctypes.c_int32),
                ("rhs_rows_per_strip", ctypes.c_int32),
                ("zsweep_columns_per_lane", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def load(path=LIB_PATH):
    """Load libfsei.so (once) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FseiUnavailable("libfsei.so not built at %s (run __graft_entry__.build())" % path)
    try:
        lib = ctypes.CDLL(path)
    except OSError as exc:
        raise FseiUnavailable("cannot load %s: %s" % (path, exc)) from exc
    vp = ctypes.c_void_p
    lib.fsei_grid_create.argtypes = [ctypes.POINTER(GridDesc), ctypes.POINTER(vp)]
    lib.fsei_grid_create.restype = ctypes.c_int
    lib.fsei_grid_destroy.argtypes = [vp]
    lib.fsei_grid_destroy.restype = None
    lib.fsei_grid_workspace_bytes.argtypes = [vp]
    lib.fsei_grid_workspace_bytes.restype = ctypes.c_int64
    lib.fsei_step.argtypes = [vp, ctypes.POINTER(State), vp, vp, vp,
                              ctypes.POINTER(StepParams), ctypes.c_int32, vp,
                              ctypes.POINTER(StepStats)]
    lib.fsei_step.restype = ctypes.c_int
    lib.fsei_step_host.argtypes = [vp, ctypes.POINTER(State), ctypes.POINTER(State), vp, vp, vp,
                                   ctypes.POINTER(StepParams), ctypes.c_int32, vp,
                                   ctypes.POINTER(StepStats)]
    lib.fsei_step_host.restype = ctypes.c_int
    lib.fsei_step_host_join.argtypes = [vp, vp]
    lib.fsei_step_host_join.restype = ctypes.c_int
    lib.fsei_poisson_solve.argtypes = [vp, vp, vp, vp]
    lib.fsei_poisson_solve.restype = ctypes.c_int
    lib.fsei_adjoint_step.argtypes = [vp, ctypes.POINTER(State), ctypes.POINTER(StepParams),
                                      ctypes.POINTER(State), vp, vp, vp, vp]
    lib.fsei_adjoint_step.restype = ctypes.c_int
    lib.fsei_batch_create.argtypes = [ctypes.POINTER(GridDesc), ctypes.c_int32, ctypes.POINTER(vp)]
    lib.fsei_batch_create.restype = ctypes.c_int
    lib.fsei_batch_destroy.argtypes = [vp]
    lib.fsei_batch_destroy.restype = None
    lib.fsei_batch_size.argtypes = [vp]
    lib.fsei_batch_size.restype = ctypes.c_int32
    lib.fsei_batch_step.argtypes = [vp, ctypes.POINTER(State), ctypes.POINTER(vp),
                                    ctypes.POINTER(StepParams), ctypes.c_int32, vp,
                                    ctypes.POINTER(StepStats)]
    lib.fsei_batch_step.restype = ctypes.c_int
    lib.fsei_grid_check_bounds.argtypes = [vp]
    lib.fsei_grid_check_bounds.restype = ctypes.c_int
    lib.fsei_grid_poke_guard.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64]
    lib.fsei_grid_poke_guard.restype = ctypes.c_int
    lib.fsei_set_kernel_timing.argtypes = [vp, ctypes.c_int32]
    lib.fsei_set_kernel_timing.restype = ctypes.c_int
    lib.fsei_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.c_int32]
    lib.fsei_kernel_times.restype = ctypes.c_int32
    lib.fsei_kernel_name.argtypes = [ctypes.c_int32]
    lib.fsei_kernel_name.restype = ctypes.c_char_p
    lib.fsei_grid_autotune.argtypes = [vp, ctypes.c_int32, vp, ctypes.POINTER(Schedule)]
    lib.fsei_grid_autotune.restype = ctypes.c_int
    lib.fsei_grid_get_schedule.argtypes = [vp, ctypes.POINTER(Schedule)]
    lib.fsei_grid_get_schedule.restype = ctypes.c_int
    lib.fsei_grid_set_schedule.argtypes = [vp, ctypes.POINTER(Schedule)]
    lib.fsei_grid_set_schedule.restype = ctypes.c_int
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int32)
    lib.fsei_ib_forcing.argtypes = [vp, vp, vp, vp, vp, vp, vp, ctypes.c_int32, ctypes.c_double,
                                    vp, vp, vp, vp, vp, ip]
    lib.fsei_ib_forcing.restype = ctypes.c_int
    lib.fsei_ib_loads.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_int32,
                                  ctypes.c_int32, ctypes.c_double, ctypes.c_double, vp, vp, vp,
                                  ip]
    lib.fsei_ib_loads.restype = ctypes.c_int
    del dp
    lib.fsei_batch_set_max_group.argtypes = [vp, ctypes.c_int32]
    lib.fsei_batch_set_max_group.restype = ctypes.c_int
    lib.fsei_batch_launch_groups.argtypes = [vp]
    lib.fsei_batch_launch_groups.restype = ctypes.c_int32
    lib.fsei_batch_autotune.argtypes = [vp, ctypes.c_int32, vp]
    lib.fsei_batch_autotune.restype = ctypes.c_int
    lib.fsei_fp64_fma_rate.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.fsei_fp64_fma_rate.restype = ctypes.c_int
    lib.fsei_last_error.argtypes = []
    lib.fsei_last_error.restype = ctypes.c_char_p
    lib.fsei_version.argtypes = []
    lib.fsei_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status, stats=None):
    if status != FSEI_OK:
        raise FseiError(status, load().fsei_last_error().decode(), stats)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


class Grid:
    """Owning wrapper of an fsei_grid handle (fsei_grid_create /
    fsei_grid_destroy)."""

    def __init__(self, nx, ny, nz, lx, ly, zbc=FSEI_Z_WALLS, lz=2.0, stretch=0.0,
                 prec=FSEI_FP64, zfaces=None, near_zero_tau=0.0):
        lib = load()
        d = GridDesc()
        d.nx, d.ny, d.nz = nx, ny, nz
        d.lx, d.ly, d.zbc, d.lz, d.stretch = lx, ly, zbc, lz, stretch
        d.prec = prec
        d.near_zero_tau = near_zero_tau
        self._zf = None
        if zfaces is not None:
            self._zf = np.ascontiguousarray(zfaces, dtype=np.float64)
            d.zfaces = self._zf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        h = ctypes.c_void_p()
        _check(lib.fsei_grid_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self.nx, self.ny, self.nz = nx, ny, nz
        self.prec = prec

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def workspace_bytes(self):
        return load().fsei_grid_workspace_bytes(self.handle)

    def autotune(self, force=False, stream=None):
        """fsei_grid_autotune: pick the launch schedule by measurement (or
        take the one this process holds for the shape); returns it."""
        out = Schedule()
        _check(load().fsei_grid_autotune(self.handle, FSEI_TUNE_FORCE if force else 0,
                                         _stream_handle(stream), ctypes.byref(out)))
        return out.as_dict()

    @property
    def schedule(self):
        """fsei_grid_get_schedule as a dict."""
        out = Schedule()
        _check(load().fsei_grid_get_schedule(self.handle, ctypes.byref(out)))
        return out.as_dict()

    def set_schedule(self, sched):
        """fsei_grid_set_schedule from a dict (missing keys keep their
        current values)."""
        cur = self.schedule
        cur.update(sched)
        s = Schedule(**cur)
        _check(load().fsei_grid_set_schedule(self.handle, ctypes.byref(s)))

    def close(self):
        if getattr(self, "handle", None):
            load().fsei_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def grid_create(**kw):
    return Grid(**kw)


def step(grid, state, f=None, re=100.0, dt=1e-3, cfl=0.0, gamma=1.5, rho=-0.5,
         fconst=(0.0, 0.0, 0.0), nsteps=1, stream=None, stats=True, scheme=FSEI_AB2_CN,
         rheology=None):
    """fsei_step on a dict of torch tensors u, v, w, p, hu, hv, hw and the
    key have_prev_h (updated in place).  f: None or (fx, fy, fz) tensors.
    scheme: FSEI_AB2_CN (Eq. 3) or FSEI_RK3_CN (three sub-steps per step).
    rheology: None (Newtonian) or a dict lam, n, a, eta_inf (Carreau-Yasuda).
    Returns the statistics dict of the last step when stats=True (the call
    then synchronises the stream), else None."""
    lib = load()
    st = State(_ptr(state["u"]), _ptr(state["v"]), _ptr(state["w"]), _ptr(state["p"]),
               _ptr(state["hu"]), _ptr(state["hv"]), _ptr(state["hw"]),
               int(state.get("have_prev_h", 0)))
    rh, cy = _rheology(rheology)
    prm = StepParams(re, dt, cfl, gamma, rho, (ctypes.c_double * 3)(*fconst), int(scheme), rh, cy)
    fx, fy, fz = (None, None, None) if f is None else f
    out = StepStats() if stats else None
    status = lib.fsei_step(grid.handle, ctypes.byref(st), _ptr(fx), _ptr(fy), _ptr(fz),
                           ctypes.byref(prm), int(nsteps), _stream_handle(stream),
                           ctypes.byref(out) if out is not None else None)
    state["have_prev_h"] = st.have_prev_h
    res = out.as_dict() if out is not None else None
    _check(status, res)
    return res


def step_host(grid, host, dev, f=None, re=100.0, dt=1e-3, cfl=0.0, gamma=1.5, rho=-0.5,
              fconst=(0.0, 0.0, 0.0), nsteps=1, stream=None, stats=True, scheme=FSEI_AB2_CN,
              rheology=None):
    """fsei_step_host: host is a dict of CPU tensors u, v, w, p, hu, hv, hw
    (pinned for asynchronous copies) and the key have_prev_h (updated in
    place); dev a dict of device tensors of the same shapes, the staging
    state.  With stats=True the call waits for the copies back and returns
    the statistics dict; else the copies back finish on the grid's copy
    stream (step_host_join orders a stream after them)."""
    lib = load()

    def st_of(d, have):
        return State(_ptr(d["u"]), _ptr(d["v"]), _ptr(d["w"]), _ptr(d["p"]),
                     _ptr(d["hu"]), _ptr(d["hv"]), _ptr(d["hw"]), have)
    hs = st_of(host, int(host.get("have_prev_h", 0)))
    ds = st_of(dev, 0)
    rh, cy = _rheology(rheology)
    prm = StepParams(re, dt, cfl, gamma, rho, (ctypes.c_double * 3)(*fconst), int(scheme), rh, cy)
    fx, fy, fz = (None, None, None) if f is None else f
    out = StepStats() if stats else None
    status = lib.fsei_step_host(grid.handle, ctypes.byref(hs), ctypes.byref(ds), _ptr(fx),
                                _ptr(fy), _ptr(fz), ctypes.byref(prm), int(nsteps),
                                _stream_handle(stream),
                                ctypes.byref(out) if out is not None else None)
    host["have_prev_h"] = hs.have_prev_h
    res = out.as_dict() if out is not None else None
    _check(status, res)
    return res


def step_host_join(grid, stream=None):
    """fsei_step_host_join: order the stream after the last step_host call's
    copies back."""
    _check(load().fsei_step_host_join(grid.handle, _stream_handle(stream)))


def poisson_solve(grid, rhs, phi, stream=None):
    """fsei_poisson_solve: phi with D G phi = rhs (device tensors)."""
    _check(load().fsei_poisson_solve(grid.handle, _ptr(rhs), _ptr(phi),
                                     _stream_handle(stream)))


def adjoint_step(grid, fwd, adj, fbar=None, re=100.0, dt=1e-3, gamma=1.5, rho=-0.5,
                 fconst=(0.0, 0.0, 0.0), stream=None):
    """fsei_adjoint_step.  fwd: dict with the step's input u, v, w (and
    have_prev_h); adj: dict of cotangent tensors u, v, w, p, hu, hv, hw,
    updated in place from output to input cotangents; fbar: None or
    (fbx, fby, fbz) accumulated in place."""
    lib = load()
    f = State(_ptr(fwd["u"]), _ptr(fwd["v"]), _ptr(fwd["w"]), None, None, None, None,
              int(fwd.get("have_prev_h", 0)))
    a = State(_ptr(adj["u"]), _ptr(adj["v"]), _ptr(adj["w"]), _ptr(adj["p"]),
              _ptr(adj["hu"]), _ptr(adj["hv"]), _ptr(adj["hw"]), 0)
    prm = StepParams(re, dt, 0.0, gamma, rho, (ctypes.c_double * 3)(*fconst))
    fb = (None, None, None) if fbar is None else fbar
    _check(lib.fsei_adjoint_step(grid.handle, ctypes.byref(f), ctypes.byref(prm),
                                 ctypes.byref(a), _ptr(fb[0]), _ptr(fb[1]), _ptr(fb[2]),
                                 _stream_handle(stream)))


def _desc(nx, ny, nz, lx, ly, zbc=FSEI_Z_WALLS, lz=2.0, stretch=0.0, prec=FSEI_FP64,
          near_zero_tau=0.0):
    d = GridDesc()
    d.nx, d.ny, d.nz = nx, ny, nz
    d.lx, d.ly, d.zbc, d.lz, d.stretch = lx, ly, zbc, lz, stretch
    d.prec = prec
    d.near_zero_tau = near_zero_tau
    return d


class Batch:
    """Owning wrapper of an fsei_batch (fsei_batch_create / destroy).
    boxes: list of dicts with the fsei.Grid keyword arguments."""

    def __init__(self, boxes):
        lib = load()
        arr = (GridDesc * len(boxes))(*[_desc(**b) for b in boxes])
        h = ctypes.c_void_p()
        _check(lib.fsei_batch_create(arr, len(boxes), ctypes.byref(h)))
        self.handle = h
        self.n = len(boxes)

    def autotune(self, force=False, stream=None):
        """fsei_batch_autotune: one measured schedule per distinct box shape,
        refined for shapes shared by several boxes by timing their grouped
        launches."""
        _check(load().fsei_batch_autotune(self.handle, FSEI_TUNE_FORCE if force else 0,
                                          _stream_handle(stream)))

    def set_max_group(self, max_boxes):
        """fsei_batch_set_max_group: boxes per launch group (0: no limit)."""
        _check(load().fsei_batch_set_max_group(self.handle, int(max_boxes)))

    @property
    def launch_groups(self):
        """fsei_batch_launch_groups: launch groups of the last capture."""
        return load().fsei_batch_launch_groups(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            load().fsei_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_step(batch, states, forces, params, nsteps=1, stream=None, stats=True):
    """fsei_batch_step.  states: list of state dicts (as for step); forces:
    None or list of None / (fx, fy, fz); params: list of dicts with re, dt,
    cfl, gamma, rho, fconst and optionally scheme.  Returns the per-box
    statistics when stats."""
    lib = load()
    n = batch.n
    st = (State * n)()
    for i, s in enumerate(states):
        st[i] = State(_ptr(s["u"]), _ptr(s["v"]), _ptr(s["w"]), _ptr(s["p"]), _ptr(s["hu"]),
                      _ptr(s["hv"]), _ptr(s["hw"]), int(s.get("have_prev_h", 0)))
    fp = None
    if forces is not None:
        fp = (ctypes.c_void_p * (3 * n))()
        for i, f in enumerate(forces):
            for c in range(3):
                fp[3 * i + c] = None if f is None else f[c].data_ptr()
    prm = (StepParams * n)()
    for i, p in enumerate(params):
        prm[i] = StepParams(p.get("re", 100.0), p.get("dt", 0.0), p.get("cfl", 0.0),
                            p.get("gamma", 1.5), p.get("rho", -0.5),
                            (ctypes.c_double * 3)(*p.get("fconst", (0.0, 0.0, 0.0))),
                            int(p.get("scheme", FSEI_AB2_CN)), *_rheology(p.get("rheology")))
    out = (StepStats * n)() if stats else None
    status = lib.fsei_batch_step(batch.handle, st, fp, prm, int(nsteps), _stream_handle(stream),
                                 out)
    for i, s in enumerate(states):
        s["have_prev_h"] = st[i].have_prev_h
    res = [o.as_dict() for o in out] if out is not None else None
    _check(status, res)
    return res


def ib_forcing(grid, vel, markers, dt, f, u_at=None, stream=None):
    """fsei_ib_forcing.  vel: (u, v, w) device tensors; markers: dict of
    device float64 tensors xb (M x 3), ub (M x 3), dvb (M); f: (fx, fy, fz)
    device tensors the force is added to; u_at: None or a device (M x 3)
    float64 tensor for the interpolated velocity.  Returns the number of
    skipped markers (the call synchronises)."""
    n = int(markers["xb"].shape[0])
    sk = ctypes.c_int32(0)
    _check(load().fsei_ib_forcing(grid.handle, _ptr(vel[0]), _ptr(vel[1]), _ptr(vel[2]),
                                  _ptr(markers["xb"]), _ptr(markers["ub"]), _ptr(markers["dvb"]),
                                  n, float(dt), _ptr(f[0]), _ptr(f[1]), _ptr(f[2]), _ptr(u_at),
                                  _stream_handle(stream), ctypes.byref(sk)))
    return sk.value


def ib_loads(grid, p, vel, surface, probe, re, node_force=None, stream=None):
    """fsei_ib_loads.  surface: dict of device tensors xf, nf (F x 3 float64),
    af (F, float64), optionally two_sided (F, int32) and tris (F x 3, int32)
    with nnodes; node_force: None or an (nnodes x 3) float64 tensor added to.
    Returns (face_force (F x 3 device tensor), skipped faces, bad node
    indices)."""
    import torch
    nf = int(surface["xf"].shape[0])
    ff = torch.empty((nf, 3), dtype=torch.float64, device=surface["xf"].device)
    sk = (ctypes.c_int32 * 2)()
    _check(load().fsei_ib_loads(grid.handle, _ptr(p), _ptr(vel[0]), _ptr(vel[1]), _ptr(vel[2]),
                                _ptr(surface["xf"]), _ptr(surface["nf"]), _ptr(surface["af"]),
                                _ptr(surface.get("two_sided")), _ptr(surface.get("tris")), nf,
                                int(surface.get("nnodes", 0)), float(probe), float(re), _ptr(ff),
                                _ptr(node_force), _stream_handle(stream), sk))
    return ff, sk[0], sk[1]


def check_bounds(grid):
    """fsei_grid_check_bounds: raises FseiError(FSEI_E_BOUNDS) if a guard
    zone of a grid created with FSEI_CHECK_BOUNDS=1 was written."""
    _check(load().fsei_grid_check_bounds(grid.handle))


def poke_guard(grid, buffer, side, offset):
    """fsei_grid_poke_guard: change one guard byte of a grid in the
    bounds-checking mode (for tests of the detector)."""
    _check(load().fsei_grid_poke_guard(grid.handle, int(buffer), int(side), int(offset)))


def set_kernel_timing(grid, enable):
    """fsei_set_kernel_timing: event pairs around every kernel launch."""
    _check(load().fsei_set_kernel_timing(grid.handle, int(bool(enable))))


def kernel_times(grid):
    """fsei_kernel_times: {kernel name: (total ms, launches)} since the last
    call (synchronises the device)."""
    lib = load()
    cap = 32
    ms = (ctypes.c_double * cap)()
    n = (ctypes.c_int64 * cap)()
    count = lib.fsei_kernel_times(grid.handle, ms, n, cap)
    return {lib.fsei_kernel_name(k).decode(): (ms[k], n[k]) for k in range(count)}


def fp64_fma_rate(stream=None):
    """fsei_fp64_fma_rate: measured DFMA throughput of the current device,
    in 10^9 thread instructions per second."""
    out = ctypes.c_double()
    _check(load().fsei_fp64_fma_rate(_stream_handle(stream), ctypes.byref(out)))
    return out.value


def version():
    return load().fsei_version().decode()
