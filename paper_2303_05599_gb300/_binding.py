"""ctypes binding of ``libglasma_gb300.so`` (declared in include/glasma.h).

Argument marshalling only: every numerical step runs in the library's CUDA
kernels.  PyTorch supplies the device workspace and the CUDA stream.  Loading
fails loudly when the library is missing; there is no other code path.
"""
import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libglasma_gb300.so")

GL_MAX_SPECIES = 8
GL_OK, GL_ERR_ARG, GL_ERR_CUDA, GL_ERR_STATE, GL_ERR_TIMEOUT, GL_ERR_NUMERIC, GL_ERR_SIZE = range(7)
GL_FP64, GL_FP32_2ROW = 0, 1
(GL_BUF_LINKS, GL_BUF_PHI, GL_BUF_E, GL_BUF_PI, GL_BUF_SITE, GL_BUF_PARTICLES, GL_BUF_JETS, GL_BUF_ENERGY,
 GL_BUF_PTAU) = range(9)
JET_LEN = 44
GL_NATIVE_FIELDS, GL_NATIVE_PARTICLES = 0, 1
GL_CFG_PTAU_DIAGNOSTIC = 1

STATUS_NAMES = {0: "GL_OK", 1: "GL_ERR_ARG", 2: "GL_ERR_CUDA", 3: "GL_ERR_STATE", 4: "GL_ERR_TIMEOUT",
                5: "GL_ERR_NUMERIC", 6: "GL_ERR_SIZE"}


class gl_config(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("Ns", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("reunit_every", ctypes.c_int32), ("L_fm", ctypes.c_double), ("g2mu_GeV", ctypes.c_double),
                ("mIR_GeV", ctypes.c_double), ("LambdaUV_GeV", ctypes.c_double),
                ("dtau_over_a", ctypes.c_double), ("seed", ctypes.c_uint64), ("sort_every", ctypes.c_int32),
                ("n_jets", ctypes.c_int32), ("flags", ctypes.c_uint32), ("reserved", ctypes.c_int32)]


class gl_species(ctypes.Structure):
    _fields_ = [("mass_GeV", ctypes.c_double), ("tau_form_fm", ctypes.c_double), ("count", ctypes.c_int64),
                ("rep", ctypes.c_int32), ("mom_mode", ctypes.c_int32), ("p0_GeV", ctypes.c_double),
                ("p1_GeV", ctypes.c_double)]


_D8 = ctypes.c_double * GL_MAX_SPECIES


class gl_obs(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("tau_fm", ctypes.c_double), ("n_species", ctypes.c_int32),
                ("what", ctypes.c_uint32), ("n_active", ctypes.c_int64 * GL_MAX_SPECIES),
                ("sum_px2", _D8), ("sum_py2", _D8), ("sum_pL2", _D8), ("sum_dpT2", _D8),
                ("casimir2_dev", _D8), ("casimir3_dev", _D8), ("gauss_max", ctypes.c_double),
                ("gauss_rms", ctypes.c_double), ("unitarity_max", ctypes.c_double),
                ("mean_trE_T2", ctypes.c_double), ("mean_trE_L2", ctypes.c_double),
                ("mean_trB_T2", ctypes.c_double), ("mean_trB_L2", ctypes.c_double)]


# every symbol include/glasma.h declares, with its signature
_P = ctypes.c_void_p
SIGNATURES = {
    "gl_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(gl_config), ctypes.POINTER(gl_species), ctypes.c_int32]),
    "gl_create": (ctypes.c_int, [ctypes.POINTER(gl_config), ctypes.POINTER(gl_species), ctypes.c_int32, _P,
                                 ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    "gl_destroy": (ctypes.c_int, [_P]),
    "gl_error_string": (ctypes.c_char_p, [_P]),
    "glasma_init": (ctypes.c_int, [_P]),
    "wong_init": (ctypes.c_int, [_P]),
    "gl_upload": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t]),
    "gl_download": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t]),
    "gl_set_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "gl_native_bytes": (ctypes.c_size_t, [_P, ctypes.c_int]),
    "gl_download_native": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t]),
    "gl_upload_native": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t]),
    "glasma_step": (ctypes.c_int, [_P, ctypes.c_int32]),
    "wong_site_fields": (ctypes.c_int, [_P]),
    "wong_push": (ctypes.c_int, [_P]),
    "gl_step_coupled": (ctypes.c_int, [_P, ctypes.c_int32]),
    "observables": (ctypes.c_int, [_P, ctypes.POINTER(gl_obs)]),
    "gl_observables_ex": (ctypes.c_int, [_P, ctypes.c_uint32, ctypes.POINTER(gl_obs)]),
    "gl_autotune": (ctypes.c_int, [_P, _P, _P]),
    "gl_tuning": (ctypes.c_int, [_P, _P, _P]),
    "gl_jets_observables": (ctypes.c_int, [_P, _P]),
    "gl_ensemble_sums_noalloc": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, _P, _P, _P, ctypes.c_uint32,
                                                ctypes.c_double, _P, _P]),
    "gl_batch_workspace_bytes": (ctypes.c_size_t, [_P, _P, ctypes.c_int32, ctypes.c_int32]),
    "gl_batch_create": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_size_t, _P,
                                       ctypes.POINTER(_P)]),
    "gl_batch_destroy": (ctypes.c_int, [_P]),
    "gl_batch_error_string": (ctypes.c_char_p, [_P]),
    "gl_batch_event": (_P, [_P, ctypes.c_int32]),
    "gl_batch_init": (ctypes.c_int, [_P]),
    "gl_batch_autotune": (ctypes.c_int, [_P, _P, _P]),
    "gl_batch_tuning": (ctypes.c_int, [_P, _P, _P, _P]),
    "gl_batch_step": (ctypes.c_int, [_P, ctypes.c_int32]),
    "gl_batch_step_timed": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "gl_batch_observables": (ctypes.c_int, [_P, _P]),
    "gl_batch_upload": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "gl_batch_upload_native": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "gl_batch_set_launch": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32]),
    "gl_batch_get_launch": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "gl_batch_observables_ex": (ctypes.c_int, [_P, ctypes.c_uint32, _P]),
    "gl_batch_observables_begin": (ctypes.c_int, [_P, ctypes.c_uint32]),
    "gl_batch_observables_end": (ctypes.c_int, [_P, _P]),
    "gl_batch_obs_row_bytes": (ctypes.c_size_t, []),
    "gl_batch_segment_rows": (ctypes.c_int32, [_P]),
    "gl_batch_set_segment_rows": (ctypes.c_int, [_P, ctypes.c_int32]),
}

GL_NOALLOC_MAX_PARTICLES = 2097152
GL_OBS_PARTICLES, GL_OBS_FIELDS, GL_OBS_ALL = 1, 2, 3
BATCH_TILES = ("32x8", "32x4", "32x16")   # FP64 field tiles of a batch (32x4 is the one used)
# FP32 field launch shapes of the strip kernel: resident warps per SM
STRIP_SHAPES = ("strip16", "strip12", "strip8")


def _shape_names(precision):
    return BATCH_TILES if precision == 0 else STRIP_SHAPES

_lib = None


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libglasma_gb300.so is not built; run __graft_entry__.build() "
                               "(python paper_2303_05599_gb300/build.py)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class GlasmaError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__("%s: %s (%s)" % (where, STATUS_NAMES.get(status, status), msg))
        self.status = status


def _check(status, ctx, where):
    if status != GL_OK:
        msg = lib().gl_error_string(ctx)
        raise GlasmaError(status, where, msg.decode() if msg else "")


def make_config(w):
    """gl_config from a workloads.Workload."""
    return gl_config(N=w.N, Ns=w.Ns, precision=w.precision, reunit_every=w.reunit_every, L_fm=w.L_fm,
                     g2mu_GeV=w.g2mu_GeV, mIR_GeV=w.mIR_GeV, LambdaUV_GeV=w.LambdaUV_GeV,
                     dtau_over_a=w.dtau_over_a, seed=w.seed, sort_every=w.sort_every, n_jets=w.n_jets,
                     flags=GL_CFG_PTAU_DIAGNOSTIC if w.ptau_diagnostic else 0, reserved=0)


def make_species(w):
    arr = (gl_species * max(1, len(w.species)))()
    for k, s in enumerate(w.species):
        arr[k] = gl_species(mass_GeV=s.mass_GeV, tau_form_fm=s.tau_form_fm, count=s.count, rep=s.rep,
                            mom_mode=s.mom_mode, p0_GeV=s.p0_GeV, p1_GeV=s.p1_GeV)
    return arr


def gl_workspace_bytes(w):
    cfg = make_config(w)
    sp = make_species(w)
    return int(lib().gl_workspace_bytes(ctypes.byref(cfg), sp, len(w.species)))


class Event:
    """One MV event with its particle ensemble on the current CUDA device.

    The workspace is a torch uint8 tensor on the device; all calls are
    enqueued on the given torch stream (default: the current stream)."""

    def __init__(self, workload, stream=None, device=None):
        import torch
        self.w = workload
        self.cfg = make_config(workload)
        self.sp = make_species(workload)
        nbytes = int(lib().gl_workspace_bytes(ctypes.byref(self.cfg), self.sp, len(workload.species)))
        if nbytes == 0:
            raise GlasmaError(GL_ERR_ARG, "gl_workspace_bytes", "invalid workload")
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.ctx = ctypes.c_void_p()
        st = lib().gl_create(ctypes.byref(self.cfg), self.sp, len(workload.species), ctypes.c_void_p(aligned),
                             nbytes, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.ctx))
        _check(st, None, "gl_create")
        self.N = workload.N
        self.np = workload.n_particles
        self.n_jets = workload.n_jets

    @classmethod
    def view(cls, ctx, workload):
        """An Event over a context owned by someone else (a batch)."""
        ev = cls.__new__(cls)
        ev.w = workload
        ev.ctx = ctypes.c_void_p(ctx)
        ev.N = workload.N
        ev.np = workload.n_particles
        ev.n_jets = workload.n_jets
        ev.owned = False
        return ev

    def close(self):
        if self.ctx and getattr(self, "owned", True):
            lib().gl_destroy(self.ctx)
        self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- the C ABI, one call each
    def glasma_init(self):
        _check(lib().glasma_init(self.ctx), self.ctx, "glasma_init")

    def wong_init(self):
        _check(lib().wong_init(self.ctx), self.ctx, "wong_init")

    def glasma_step(self, n=1):
        _check(lib().glasma_step(self.ctx, n), self.ctx, "glasma_step")

    def wong_site_fields(self):
        _check(lib().wong_site_fields(self.ctx), self.ctx, "wong_site_fields")

    def wong_push(self):
        _check(lib().wong_push(self.ctx), self.ctx, "wong_push")

    def step(self, n=1):
        _check(lib().gl_step_coupled(self.ctx, n), self.ctx, "gl_step_coupled")

    def set_step(self, n):
        _check(lib().gl_set_step(self.ctx, n), self.ctx, "gl_set_step")

    def observables(self, what=None):
        """gl_obs of the current time; `what` (GL_OBS_* bits) selects the parts
        computed, all by default."""
        o = gl_obs()
        if what is None:
            _check(lib().observables(self.ctx, ctypes.byref(o)), self.ctx, "observables")
        else:
            _check(lib().gl_observables_ex(self.ctx, what, ctypes.byref(o)), self.ctx, "gl_observables_ex")
        return o

    def autotune(self):
        t = ctypes.c_int32()
        p = ctypes.c_int32()
        _check(lib().gl_autotune(self.ctx, ctypes.byref(t), ctypes.byref(p)), self.ctx, "gl_autotune")
        f = (ctypes.c_float * 4)()
        q = (ctypes.c_float * 3)()
        lib().gl_tuning(self.ctx, f, q)
        names = ("32x8", "32x4", "32x2", "32x16") if self.w.precision == 0 else STRIP_SHAPES + ("strip16",)
        return {"tile": names[t.value], "push_block": p.value,
                "field_ms": list(f), "push_ms": list(q)}

    def _shape(self, which):
        V = self.N * self.N
        return {GL_BUF_LINKS: (2, V, 18), GL_BUF_PHI: (V, 8), GL_BUF_E: (2, V, 8), GL_BUF_PI: (V, 8),
                GL_BUF_SITE: (6, V, 8), GL_BUF_PARTICLES: (self.np, 16),
                GL_BUF_JETS: (self.n_jets, JET_LEN), GL_BUF_ENERGY: (V,), GL_BUF_PTAU: (self.np,)}[which]

    def jets_observables(self):
        """Mean over the jet-correlator probes of X_i . X_i (i = x, y, z), GeV^2."""
        out = (ctypes.c_double * 3)()
        _check(lib().gl_jets_observables(self.ctx, out), self.ctx, "gl_jets_observables")
        return list(out)

    def upload(self, which, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64)
        if a.shape != self._shape(which) and a.size == int(np.prod(self._shape(which))):
            a = a.reshape(self._shape(which))
        _check(lib().gl_upload(self.ctx, which, a.ctypes.data_as(ctypes.c_void_p), a.size), self.ctx, "gl_upload")

    def download(self, which):
        a = np.empty(self._shape(which), dtype=np.float64)
        _check(lib().gl_download(self.ctx, which, a.ctypes.data_as(ctypes.c_void_p), a.size), self.ctx,
               "gl_download")
        return a

    def native_bytes(self, part):
        """Size of native snapshot part GL_NATIVE_FIELDS or GL_NATIVE_PARTICLES."""
        return int(lib().gl_native_bytes(self.ctx, part))

    def download_native(self, part, out=None):
        """Native snapshot part (device layout bytes, gl_download_native) into a
        new uint8 array, or into `out` (a C-contiguous array of exactly
        native_bytes(part) bytes, e.g. the numpy view of a pinned tensor)."""
        n = self.native_bytes(part)
        a = np.empty(n, dtype=np.uint8) if out is None else out
        if a.nbytes != n or not a.flags.c_contiguous:
            raise ValueError("native part %d needs a contiguous buffer of %d bytes" % (part, n))
        _check(lib().gl_download_native(self.ctx, part, a.ctypes.data_as(ctypes.c_void_p), n), self.ctx,
               "gl_download_native")
        return a

    def upload_native(self, part, arr):
        """Native snapshot part from a C-contiguous buffer (gl_upload_native)."""
        a = np.ascontiguousarray(arr)
        _check(lib().gl_upload_native(self.ctx, part, a.ctypes.data_as(ctypes.c_void_p), a.nbytes), self.ctx,
               "gl_upload_native")


class Batch:
    """Many MV events (same precision and time step, any N) advanced together
    by one field launch and one push launch per step, replayed from a CUDA
    graph.  The workspace is one torch uint8 tensor; the stream must not be
    the default stream."""

    def __init__(self, workloads, stream=None, device=None):
        import torch
        self.ws_list = list(workloads)
        ne = len(self.ws_list)
        ns = max(len(w.species) for w in self.ws_list)
        if any(len(w.species) != ns for w in self.ws_list):
            raise GlasmaError(GL_ERR_ARG, "Batch", "every event needs the same number of species")
        self.cfgs = (gl_config * ne)(*[make_config(w) for w in self.ws_list])
        sp = (gl_species * max(1, ne * ns))()
        for e, w in enumerate(self.ws_list):
            for k, s_ in enumerate(w.species):
                sp[e * ns + k] = gl_species(mass_GeV=s_.mass_GeV, tau_form_fm=s_.tau_form_fm, count=s_.count,
                                            rep=s_.rep, mom_mode=s_.mom_mode, p0_GeV=s_.p0_GeV, p1_GeV=s_.p1_GeV)
        self.sp = sp
        nbytes = int(lib().gl_batch_workspace_bytes(self.cfgs, sp, ns, ne))
        if nbytes == 0:
            raise GlasmaError(GL_ERR_ARG, "gl_batch_workspace_bytes", "invalid batch")
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        aligned = (self.workspace.data_ptr() + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self.b = ctypes.c_void_p()
        st = lib().gl_batch_create(self.cfgs, sp, ns, ne, ctypes.c_void_p(aligned), nbytes,
                                   ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self.b))
        _check(st, None, "gl_batch_create")
        self.ne = ne
        self.events = [Event.view(lib().gl_batch_event(self.b, e), self.ws_list[e]) for e in range(ne)]

    def _chk(self, st, where):
        if st != GL_OK:
            msg = lib().gl_batch_error_string(self.b)
            raise GlasmaError(st, where, msg.decode() if msg else "")

    def init(self):
        self._chk(lib().gl_batch_init(self.b), "gl_batch_init")

    def autotune(self):
        t = ctypes.c_int32()
        p = ctypes.c_int32()
        self._chk(lib().gl_batch_autotune(self.b, ctypes.byref(t), ctypes.byref(p)), "gl_batch_autotune")
        f = (ctypes.c_float * 3)()
        q = (ctypes.c_float * 3)()
        st = (ctypes.c_float * 8)()
        lib().gl_batch_tuning(self.b, f, q, st)
        out = self.launch()
        out.update({"field_ms": list(f), "push_ms": list(q), "step_ms_two_streams": st[0],
                    "step_ms_fused_by_chunk": list(st)[1:4],
                    "step_ms_push_grid_by_tile": {"1": list(st)[4:6], "2": list(st)[6:8]}})
        return out

    def launch(self):
        """The launch shapes and schedule in use."""
        v = [ctypes.c_int32() for _ in range(5)]
        self._chk(lib().gl_batch_get_launch(self.b, *[ctypes.byref(x) for x in v]), "gl_batch_get_launch")
        return {"tile": _shape_names(self.ws_list[0].precision)[v[0].value], "push_block": v[1].value,
                "push_chunk": v[2].value, "segment_rows": int(lib().gl_batch_segment_rows(self.b)),
                "fused": bool(v[3].value), "push_grid": v[4].value}

    def set_launch(self, tile, push_block=128, push_chunk=1024, fused=False, push_grid=0):
        """Fix the launch shapes and schedule (field shape: a name from
        STRIP_SHAPES for FP32 batches, from BATCH_TILES for FP64 ones)."""
        names = _shape_names(self.ws_list[0].precision)
        if tile not in names:
            raise GlasmaError(GL_ERR_ARG, "set_launch", "field shape %r is not one of %s" % (tile, names))
        self._chk(lib().gl_batch_set_launch(self.b, names.index(tile), push_block, push_chunk, int(fused),
                                            push_grid), "gl_batch_set_launch")

    def set_segment_rows(self, rows):
        """FP32: rows per strip segment of the field kernel for the current
        launch shape (0: the cost model's choice)."""
        self._chk(lib().gl_batch_set_segment_rows(self.b, rows), "gl_batch_set_segment_rows")

    def step(self, n=1):
        self._chk(lib().gl_batch_step(self.b, n), "gl_batch_step")

    def step_timed(self, n):
        """n steps with per-kernel CUDA events; returns (field_ms, push_ms) summed."""
        f = ctypes.c_double()
        p = ctypes.c_double()
        self._chk(lib().gl_batch_step_timed(self.b, n, ctypes.byref(f), ctypes.byref(p)), "gl_batch_step_timed")
        return f.value, p.value

    def upload(self, which, arrays):
        """Buffer `which` of every event from arrays[e] (canonical layout),
        with one wait for all events (gl_batch_upload)."""
        keep = []
        for ev, arr in zip(self.events, arrays):
            a = np.ascontiguousarray(arr, dtype=np.float64)
            if a.size != int(np.prod(ev._shape(which))):
                raise ValueError("array for buffer %d has %d doubles, the event needs %d"
                                 % (which, a.size, int(np.prod(ev._shape(which)))))
            keep.append(a)
        if len(keep) != self.ne:
            raise ValueError("one array per event")
        ptrs = (ctypes.c_void_p * self.ne)(*[a.ctypes.data for a in keep])
        counts = (ctypes.c_size_t * self.ne)(*[a.size for a in keep])
        self._chk(lib().gl_batch_upload(self.b, which, ptrs, counts), "gl_batch_upload")

    def upload_native(self, part, arrays):
        """Native snapshot part of every event from arrays[e] (C-contiguous,
        e.g. from Event.download_native), with one wait for all events
        (gl_batch_upload_native)."""
        keep = [np.ascontiguousarray(a) for a in arrays]
        if len(keep) != self.ne:
            raise ValueError("one array per event")
        ptrs = (ctypes.c_void_p * self.ne)(*[a.ctypes.data for a in keep])
        sizes = (ctypes.c_size_t * self.ne)(*[a.nbytes for a in keep])
        self._chk(lib().gl_batch_upload_native(self.b, part, ptrs, sizes), "gl_batch_upload_native")

    def observables(self, what=None):
        out = (gl_obs * self.ne)()
        if what is None:
            self._chk(lib().gl_batch_observables(self.b, out), "gl_batch_observables")
        else:
            self._chk(lib().gl_batch_observables_ex(self.b, what, out), "gl_batch_observables_ex")
        return list(out)

    def observables_begin(self, what=None):
        """Enqueue the observables of the current state (no wait)."""
        self._chk(lib().gl_batch_observables_begin(self.b, GL_OBS_ALL if what is None else what),
                  "gl_batch_observables_begin")

    def observables_end(self):
        """The results of the oldest outstanding observables_begin (waits)."""
        out = (gl_obs * self.ne)()
        self._chk(lib().gl_batch_observables_end(self.b, out), "gl_batch_observables_end")
        return list(out)

    def close(self):
        if self.b:
            for ev in self.events:
                ev.ctx = ctypes.c_void_p()
            lib().gl_batch_destroy(self.b)
            self.b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
