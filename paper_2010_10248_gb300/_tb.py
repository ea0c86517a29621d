"""ctypes binding of libtb.so with the C ABI's names (include/tb.h).

Argument marshalling only: every step of the propagation runs in the CUDA
library.  Array arguments may be torch tensors (host or CUDA), numpy arrays,
or raw integer addresses; streams may be a torch.cuda.Stream, an integer
cudaStream_t, or None (the legacy default stream).  There is no fallback: if
libtb.so is missing or fails to load, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtb.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "tb.h")

TB_OK, TB_EINVAL, TB_ENOMEM, TB_ECUDA, TB_EUNSTABLE, TB_ETIMEOUT, TB_EDIVERGED, TB_ESTATE = range(8)
STATUS_NAMES = {0: "TB_OK", 1: "TB_EINVAL", 2: "TB_ENOMEM", 3: "TB_ECUDA", 4: "TB_EUNSTABLE",
                5: "TB_ETIMEOUT", 6: "TB_EDIVERGED", 7: "TB_ESTATE"}
TB_ACOUSTIC, TB_TTI, TB_ELASTIC = 0, 1, 2
TB_ONESTEP, TB_BLOCKED = 0, 1
TB_F32, TB_F16, TB_BF16, TB_F32_PLAIN = 0, 1, 2, 3
TB_CKPT_SEGMENTS, TB_CKPT_BINOMIAL = 0, 1


class TBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Options(C.Structure):
    _fields_ = [("time_tile", C.c_int), ("nbl", C.c_int), ("y_bands", C.c_int),
                ("x_chunks", C.c_int), ("profile", C.c_int), ("check_nan", C.c_int),
                ("wait_timeout_s", C.c_double), ("storage", C.c_int), ("band_ctas", C.c_int),
                ("slab_planes", C.c_int), ("tti_fused", C.c_int),
                ("stream_l1", C.c_int)]


_lib = None
_lock = threading.Lock()

_vp = C.c_void_p
_SIGS = {
    "tb_create": (C.c_int, [C.POINTER(C.c_int64), C.POINTER(C.c_double), C.c_int, C.c_int,
                            C.POINTER(Options), C.POINTER(_vp)]),
    "tb_destroy": (C.c_int, [_vp]),
    "tb_set_model": (C.c_int, [_vp, _vp, _vp, _vp, C.c_double, _vp]),
    "tb_get_dt": (C.c_double, [_vp]),
    "tb_set_sources": (C.c_int, [_vp, C.c_int, _vp, C.c_int, _vp, _vp]),
    "tb_set_receivers": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "tb_forward": (C.c_int, [_vp, C.c_int, _vp, C.c_int, _vp]),
    "tb_get_field": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "tb_get_source_points": (C.c_int, [_vp, C.POINTER(C.c_int64), _vp, _vp]),
    "tb_get_receiver_points": (C.c_int, [_vp, C.POINTER(C.c_int64), _vp, _vp, _vp]),
    "tb_workspace_bytes": (C.c_size_t, [_vp]),
    "tb_kernel_time": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "tb_last_error": (C.c_char_p, [_vp]),
    "tb_fd_weights": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "tb_cfl_dt_max": (C.c_double, [C.c_int, C.POINTER(C.c_double), C.c_double]),
    "tb_tti_dt_max": (C.c_double, [C.c_int, C.POINTER(C.c_double), C.c_double, C.c_double]),
    "tb_adjoint_gradient": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, C.c_int, _vp]),
    "tb_adjoint_gradient_ckpt": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, C.c_int, C.c_int, _vp]),
    "tb_adjoint_stats": (C.c_int, [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_size_t)]),
    "tb_batch_create": (C.c_int, [C.c_int, C.POINTER(_vp)]),
    "tb_batch_destroy": (C.c_int, [_vp]),
    "tb_batch_add": (C.c_int, [_vp, _vp, C.c_int, _vp, _vp]),
    "tb_batch_step": (C.c_int, [_vp, C.c_int, _vp]),
    "tb_batch_active": (C.c_int, [_vp]),
    "tb_batch_finished": (C.c_int, [_vp, C.POINTER(_vp), C.c_int, C.POINTER(C.c_int)]),
    "tb_plan_checkpoints": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int,
                                      C.POINTER(C.c_int64)]),
    "tb_elastic_dt_max": (C.c_double, [C.c_int, C.POINTER(C.c_double), C.c_double]),
    "tb_sponge_profile": (C.c_int, [C.c_int64, C.c_int, C.c_double, C.c_double,
                                    C.POINTER(C.c_double)]),
    "tb_ricker": (C.c_int, [C.c_double, C.c_double, C.c_int, C.c_double, C.POINTER(C.c_float)]),
    "tb_selftest_wait": (C.c_int, [C.c_double, _vp]),
    "tb_measure_peaks": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double), _vp]),
    "tb_launch_count": (C.c_uint64, []),
    "tb_plan_pipeline": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                   C.POINTER(C.c_int), C.c_int]),
    "tb_plan_wavefront": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_int]),
    "tb_source_event_layout": (C.c_int, [C.c_int64, _vp, C.c_int64, C.c_int64, _vp, _vp,
                                         C.POINTER(C.c_int64)]),
    "tb_inspect_points_noalloc": (C.c_int, [C.POINTER(C.c_int64), C.POINTER(C.c_double), C.c_int,
                                            _vp, _vp, _vp, _vp]),
}


def header_functions():
    """Names of the functions include/tb.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|double|size_t|uint64_t|const char\*)\s+(tb_\w+)\s*\(",
                                 txt, flags=re.M)))


def load(path: str | None = None):
    """Load libtb.so (built by paper_2010_10248_gb300.build).  Raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"CUDA library not built: {p} (run __graft_entry__.build())")
            lib = C.CDLL(p)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
        return _lib


def _ptr(a):
    """Address of a tensor / ndarray / int (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if hasattr(a, "ctypes"):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"cannot pass {type(a)} as a pointer")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(h, st, what):
    if st != TB_OK:
        msg = load().tb_last_error(h)
        raise TBError(st, f"{what}: {msg.decode() if msg else ''}")


def tb_create(shape, spacing, space_order, physics=TB_ACOUSTIC, opt: Options | None = None):
    n = (C.c_int64 * 3)(*[int(s) for s in shape])
    hh = (C.c_double * 3)(*[float(s) for s in spacing])
    out = _vp()
    st = load().tb_create(n, hh, int(space_order), int(physics),
                          C.byref(opt) if opt is not None else None, C.byref(out))
    if st != TB_OK:
        raise TBError(st, "tb_create")
    return out.value


def tb_destroy(h):
    return load().tb_destroy(h)


def tb_set_model(h, vp, aux=None, damp=None, dt=0.0, stream=None):
    _check(h, load().tb_set_model(h, _ptr(vp), _ptr(aux), _ptr(damp), float(dt), _stream(stream)),
           "tb_set_model")


def tb_get_dt(h):
    return load().tb_get_dt(h)


def tb_set_sources(h, nsrc, coords, nt, wavelets, stream=None):
    _check(h, load().tb_set_sources(h, int(nsrc), _ptr(coords), int(nt), _ptr(wavelets),
                                    _stream(stream)), "tb_set_sources")


def tb_set_receivers(h, nrec, coords, stream=None):
    _check(h, load().tb_set_receivers(h, int(nrec), _ptr(coords), _stream(stream)),
           "tb_set_receivers")


def tb_forward(h, nt, traces, schedule=TB_BLOCKED, stream=None):
    _check(h, load().tb_forward(h, int(nt), _ptr(traces), int(schedule), _stream(stream)),
           "tb_forward")


def tb_get_field(h, which, out, stream=None):
    _check(h, load().tb_get_field(h, int(which), _ptr(out), _stream(stream)), "tb_get_field")


def tb_get_source_points(h, lin=None, dcmp=None):
    n = C.c_int64(0)
    _check(h, load().tb_get_source_points(h, C.byref(n), _ptr(lin), _ptr(dcmp)),
           "tb_get_source_points")
    return n.value


def tb_get_receiver_points(h, lin=None, corner_id=None, corner_w=None):
    n = C.c_int64(0)
    _check(h, load().tb_get_receiver_points(h, C.byref(n), _ptr(lin), _ptr(corner_id),
                                            _ptr(corner_w)), "tb_get_receiver_points")
    return n.value


def tb_workspace_bytes(h):
    return load().tb_workspace_bytes(h)


def tb_source_event_layout(lin, n1, n2):
    """The sweep kernel's source table layout for grid points `lin` (host
    only): (ev_pair [n1 * ceil(n2/2), 2] int32, slot [npts] int32, nev)."""
    import numpy as np
    lin = np.ascontiguousarray(lin, dtype=np.int64)
    npair = (int(n2) + 1) // 2
    ev = np.zeros((int(n1) * npair, 2), dtype=np.int32)
    slot = np.zeros(max(len(lin), 1), dtype=np.int32)
    nev = C.c_int64(0)
    st = load().tb_source_event_layout(len(lin), lin.ctypes.data, int(n1), int(n2), ev.ctypes.data,
                                       slot.ctypes.data, C.byref(nev))
    if st != 0:
        raise TBError(st, "tb_source_event_layout")
    return ev, slot[:len(lin)], nev.value


def tb_plan_pipeline(n1, n2, space_order, time_tile, n_tiles, cap):
    """The pipelined blocked sweep's passes as an int array [npass, 7]: launch,
    time tile, first / end owned row, first computed row, tile rows, first
    CTA (host only, no GPU)."""
    import numpy as np
    lib = load()
    n = lib.tb_plan_pipeline(int(n1), int(n2), int(space_order), int(time_tile), int(n_tiles), int(cap), None, 0)
    if n < 0:
        raise TBError(-n, "tb_plan_pipeline: invalid arguments or cap too small")
    out = np.zeros((max(n, 1), 7), dtype=np.int32)
    lib.tb_plan_pipeline(int(n1), int(n2), int(space_order), int(time_tile), int(n_tiles), int(cap),
                         out.ctypes.data_as(C.POINTER(C.c_int)), n)
    return out[:n]


def tb_plan_wavefront(n0, slab, n_sub):
    """The TTI / elastic wavefront's items as an int array [nitem, 4]: launch,
    sub-update, first plane, end plane (host only, no GPU)."""
    import numpy as np
    lib = load()
    n = lib.tb_plan_wavefront(int(n0), int(slab), int(n_sub), None, 0)
    if n < 0:
        raise TBError(-n, "tb_plan_wavefront: invalid arguments")
    out = np.zeros((max(n, 1), 4), dtype=np.int32)
    lib.tb_plan_wavefront(int(n0), int(slab), int(n_sub), out.ctypes.data_as(C.POINTER(C.c_int)), n)
    return out[:n]


def tb_kernel_time(h, kind=0):
    n = C.c_int(0)
    ms = C.c_double(0.0)
    _check(h, load().tb_kernel_time(h, int(kind), C.byref(n), C.byref(ms)), "tb_kernel_time")
    return n.value, ms.value


def tb_last_error(h):
    m = load().tb_last_error(h)
    return m.decode() if m else ""


def tb_fd_weights(space_order):
    c = (C.c_double * 16)()
    st = load().tb_fd_weights(int(space_order), c)
    if st != TB_OK:
        raise TBError(st, "tb_fd_weights")
    return [c[i] for i in range(space_order // 2 + 1)]


def tb_cfl_dt_max(space_order, spacing, vmax):
    hh = (C.c_double * 3)(*[float(s) for s in spacing])
    return load().tb_cfl_dt_max(int(space_order), hh, float(vmax))


def tb_adjoint_gradient(h, nt, residual, grad_vp=None, grad_src=None, n_snapshots=32, stream=None):
    _check(h, load().tb_adjoint_gradient(h, int(nt), _ptr(residual), _ptr(grad_vp), _ptr(grad_src),
                                         int(n_snapshots), _stream(stream)), "tb_adjoint_gradient")


def tb_adjoint_gradient_ckpt(h, nt, residual, grad_vp=None, grad_src=None, n_snapshots=32,
                             checkpointing=TB_CKPT_BINOMIAL, stream=None):
    _check(h, load().tb_adjoint_gradient_ckpt(h, int(nt), _ptr(residual), _ptr(grad_vp), _ptr(grad_src),
                                              int(n_snapshots), int(checkpointing), _stream(stream)),
           "tb_adjoint_gradient_ckpt")


def tb_adjoint_stats(h):
    """(forward steps, scratch bytes) of the handle's last adjoint gradient."""
    fs, sb = C.c_int64(0), C.c_size_t(0)
    _check(h, load().tb_adjoint_stats(h, C.byref(fs), C.byref(sb)), "tb_adjoint_stats")
    return int(fs.value), int(sb.value)


def tb_plan_checkpoints(nt, n_snapshots):
    """The binomial checkpoint schedule as an int array [nactions, 5] (kind,
    from, to, src, dst) and its forward-step count (host only, no GPU)."""
    import numpy as np
    lib = load()
    fs = C.c_int64(0)
    n = lib.tb_plan_checkpoints(int(nt), int(n_snapshots), None, 0, C.byref(fs))
    if n < 0:
        raise TBError(-n, "tb_plan_checkpoints: invalid arguments")
    out = np.zeros((max(n, 1), 5), dtype=np.int32)
    lib.tb_plan_checkpoints(int(nt), int(n_snapshots), out.ctypes.data_as(C.POINTER(C.c_int)), n, C.byref(fs))
    return out[:n], int(fs.value)


class Batch:
    """Several small acoustic shots advanced together, one launch per time
    step (tb_batch_*).  Shots are Propagator handles; traces device tensors."""

    def __init__(self, max_shots=16):
        lib = load()
        b = _vp()
        st = lib.tb_batch_create(int(max_shots), C.byref(b))
        if st != TB_OK:
            raise TBError(st, "tb_batch_create")
        self.b = b

    def add(self, h, nt, traces=None, stream=None):
        _check(h, load().tb_batch_add(self.b, h, int(nt), _ptr(traces), _stream(stream)), "tb_batch_add")

    def step(self, nsteps, stream=None):
        st = load().tb_batch_step(self.b, int(nsteps), _stream(stream))
        if st != TB_OK:
            raise TBError(st, "tb_batch_step")

    def active(self):
        return int(load().tb_batch_active(self.b))

    def finished(self, max_out=64):
        arr = (_vp * max_out)()
        n = C.c_int(0)
        st = load().tb_batch_finished(self.b, arr, int(max_out), C.byref(n))
        if st != TB_OK:
            raise TBError(st, "tb_batch_finished")
        return [arr[i] for i in range(n.value)]

    def close(self):
        if self.b:
            load().tb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tb_tti_dt_max(space_order, spacing, vmax, eps_max):
    hh = (C.c_double * 3)(*[float(s) for s in spacing])
    return load().tb_tti_dt_max(int(space_order), hh, float(vmax), float(eps_max))


def tb_elastic_dt_max(space_order, spacing, vpmax):
    hh = (C.c_double * 3)(*[float(s) for s in spacing])
    return load().tb_elastic_dt_max(int(space_order), hh, float(vpmax))


def tb_sponge_profile(n, nbl, h, vmax):
    e = (C.c_double * int(n))()
    st = load().tb_sponge_profile(int(n), int(nbl), float(h), float(vmax), e)
    if st != TB_OK:
        raise TBError(st, "tb_sponge_profile")
    return list(e)


def tb_ricker(f0, dt, nt, t0=0.0):
    out = (C.c_float * int(nt))()
    st = load().tb_ricker(float(f0), float(dt), int(nt), float(t0), out)
    if st != TB_OK:
        raise TBError(st, "tb_ricker")
    return list(out)


def tb_selftest_wait(timeout_s, stream=None):
    """Runs the bounded device-side wait on a flag nothing sets; returns the status."""
    return load().tb_selftest_wait(float(timeout_s), _stream(stream))


def tb_measure_peaks(stream=None):
    """(HBM copy GB/s, packed-FP32 FMA TFLOP/s) measured with the library's kernels."""
    hbm, fp = C.c_double(0.0), C.c_double(0.0)
    st = load().tb_measure_peaks(C.byref(hbm), C.byref(fp), _stream(stream))
    if st != TB_OK:
        raise TBError(st, "tb_measure_peaks")
    return hbm.value, fp.value


def tb_launch_count():
    return int(load().tb_launch_count())


def tb_inspect_points_noalloc(shape, spacing, npt, coords, lin, npts, stream=None):
    """Allocation-free source-point inspector; returns the status code."""
    n = (C.c_int64 * 3)(*[int(v) for v in shape])
    hh = (C.c_double * 3)(*[float(v) for v in spacing])
    return load().tb_inspect_points_noalloc(n, hh, int(npt), _ptr(coords), _ptr(lin), _ptr(npts),
                                            _stream(stream))
