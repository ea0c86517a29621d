"""GB300 temporally blocked finite-difference wave propagation with off-the-grid
sources (arXiv 2010.10248).

The computation runs in the CUDA library ``libtb.so`` (C ABI in
``include/tb.h``); ``_tb`` is its thin ctypes binding and ``Propagator`` a
convenience wrapper that keeps device buffers in torch tensors.
"""
from __future__ import annotations

from . import _tb
from ._tb import (TB_ACOUSTIC, TB_BF16, TB_BLOCKED, TB_ELASTIC, TB_F16, TB_F32, TB_F32_PLAIN, TB_ONESTEP,
                  TB_TTI, TB_CKPT_BINOMIAL, TB_CKPT_SEGMENTS, Options, TBError, load,
                  tb_adjoint_gradient, tb_adjoint_gradient_ckpt, tb_adjoint_stats, tb_plan_checkpoints,
                  tb_cfl_dt_max, tb_elastic_dt_max, tb_tti_dt_max,
                  tb_create, tb_destroy, tb_fd_weights, tb_forward, tb_get_dt, tb_get_field,
                  tb_get_receiver_points, tb_get_source_points, tb_kernel_time, tb_last_error,
                  tb_launch_count, tb_measure_peaks, tb_ricker, tb_selftest_wait, tb_set_model, tb_set_receivers, tb_set_sources,
                  tb_plan_pipeline, tb_plan_wavefront, tb_source_event_layout, tb_sponge_profile,
                  tb_workspace_bytes)

__all__ = ["Propagator", "Options", "TBError", "load", "TB_ONESTEP", "TB_BLOCKED", "TB_ACOUSTIC",
           "TB_TTI", "TB_ELASTIC", "tb_tti_dt_max", "tb_elastic_dt_max", "tb_adjoint_gradient",
           "tb_adjoint_gradient_ckpt", "tb_adjoint_stats", "tb_plan_checkpoints", "TB_CKPT_SEGMENTS",
           "TB_CKPT_BINOMIAL",
           "AcousticTraces", "TB_F32", "TB_F16", "TB_BF16", "TB_F32_PLAIN",
           "tb_create", "tb_destroy", "tb_set_model", "tb_get_dt", "tb_set_sources",
           "tb_set_receivers", "tb_forward", "tb_get_field", "tb_get_source_points",
           "tb_get_receiver_points", "tb_workspace_bytes", "tb_kernel_time", "tb_last_error",
           "tb_fd_weights", "tb_cfl_dt_max", "tb_sponge_profile", "tb_ricker", "tb_selftest_wait", "tb_measure_peaks",
           "tb_launch_count", "tb_plan_pipeline", "tb_plan_wavefront", "tb_source_event_layout"]


class Propagator:
    """One acoustic propagation problem on the current CUDA device.

    Arrays may be torch tensors (CUDA or CPU) or numpy arrays; host data are
    copied by the library.  ``forward`` returns the traces as a CUDA tensor
    [nt, nrec] unless a destination is given.
    """

    def __init__(self, shape, spacing, space_order, *, physics=TB_ACOUSTIC, time_tile=0, nbl=0,
                 y_bands=0, x_chunks=0, profile=False, check_nan=False, wait_timeout_s=0.0,
                 storage=TB_F32, band_ctas=0, slab_planes=0, tti_fused=False, stream_l1=False):
        import torch
        self._torch = torch
        opt = Options(time_tile=time_tile, nbl=nbl, y_bands=y_bands, x_chunks=x_chunks,
                      profile=int(profile), check_nan=int(check_nan),
                      wait_timeout_s=float(wait_timeout_s), storage=int(storage), band_ctas=int(band_ctas),
                      slab_planes=int(slab_planes), tti_fused=int(tti_fused),
                      stream_l1=int(stream_l1))
        self.shape = tuple(int(s) for s in shape)
        self.spacing = tuple(float(s) for s in spacing)
        self.space_order = int(space_order)
        self.physics = int(physics)
        self.storage = int(storage)
        self.h = tb_create(self.shape, self.spacing, self.space_order, self.physics, opt)
        self.nrec = 0
        self.nt_src = None

    def close(self):
        if self.h:
            tb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        return self._torch.cuda.current_stream()

    def set_model(self, vp, damp=None, dt=0.0, aux=None):
        """vp [n0, n1, n2]; aux: TTI (eps, delta, theta, phi), elastic (vs, rho),
        each [n0, n1, n2], stacked on a new leading axis (or a sequence)."""
        if aux is not None and not hasattr(aux, "data_ptr") and not hasattr(aux, "ctypes"):
            import numpy as np
            aux = np.stack([np.asarray(a, dtype=np.float32) for a in aux])
        if aux is not None and hasattr(aux, "data_ptr"):
            aux = aux.to(dtype=self._torch.float32).contiguous()
        elif aux is not None:
            import numpy as np
            aux = np.ascontiguousarray(aux, dtype=np.float32)
        tb_set_model(self.h, vp, aux, damp, dt, self._stream())
        self._aux = aux
        return self

    @property
    def dt(self):
        return tb_get_dt(self.h)

    def set_sources(self, coords, wavelets):
        coords = self._as_f64(coords)
        nsrc = coords.shape[0] if coords is not None else 0
        nt = wavelets.shape[-1] if nsrc else 0
        wav = self._as_f32(wavelets) if nsrc else None
        tb_set_sources(self.h, nsrc, coords, nt, wav, self._stream())
        self._keep = (coords, wav)  # alive until the (synchronous) call returned
        self.nt_src = nt
        return self

    def set_receivers(self, coords):
        coords = self._as_f64(coords)
        self.nrec = coords.shape[0] if coords is not None else 0
        tb_set_receivers(self.h, self.nrec, coords, self._stream())
        return self

    def forward(self, nt, traces=None, schedule=None):
        """schedule: "blocked" (time_tile steps fused per sweep; the default
        for FP32 acoustic) or "onestep" (the default for TTI, elastic and
        16-bit storage; 16-bit storage runs nothing else)."""
        torch = self._torch
        if schedule is None:
            schedule = "blocked" if self.physics == TB_ACOUSTIC and self.storage == TB_F32 else "onestep"
        sched = TB_BLOCKED if schedule == "blocked" else TB_ONESTEP
        if traces is None and self.nrec > 0:
            traces = torch.empty((nt, self.nrec), dtype=torch.float32, device="cuda")
        tb_forward(self.h, nt, traces, sched, self._stream())
        return traces

    def field(self, which=0):
        out = self._torch.empty(self.shape, dtype=self._torch.float32, device="cuda")
        tb_get_field(self.h, which, out, self._stream())
        return out

    def source_points(self):
        import numpy as np
        n = tb_get_source_points(self.h)
        lin = np.zeros(max(n, 1), dtype=np.int64)
        dcmp = np.zeros((max(self.nt_src or 0, 1), max(n, 1)), dtype=np.float32)
        tb_get_source_points(self.h, lin, dcmp)
        return lin[:n], dcmp[: (self.nt_src or 0), :n]

    def receiver_points(self):
        import numpy as np
        n = tb_get_receiver_points(self.h)
        lin = np.zeros(max(n, 1), dtype=np.int64)
        cid = np.zeros((max(self.nrec, 1), 8), dtype=np.int32)
        cw = np.zeros((max(self.nrec, 1), 8), dtype=np.float32)
        tb_get_receiver_points(self.h, lin, cid, cw)
        return lin[:n], cid[: self.nrec], cw[: self.nrec]

    def adjoint_gradient(self, nt, residual, grad_vp=None, grad_src=None, n_snapshots=32,
                         checkpointing="segments"):
        """d<traces, residual>/dvp (and /dq) for the current model and geometry.
        checkpointing: "segments" (checkpoints every ceil(nt/S) steps and a
        segment buffer) or "binomial" (exactly S stored states)."""
        torch = self._torch
        residual = residual.to(dtype=torch.float32).contiguous() if hasattr(residual, "data_ptr") else residual
        ck = {"segments": TB_CKPT_SEGMENTS, "binomial": TB_CKPT_BINOMIAL}[checkpointing]
        tb_adjoint_gradient_ckpt(self.h, nt, residual, grad_vp, grad_src, n_snapshots, ck, self._stream())
        return grad_vp, grad_src

    def adjoint_stats(self):
        """(forward steps, device scratch bytes) of the last adjoint gradient."""
        return tb_adjoint_stats(self.h)

    def kernel_time(self, kind=0):
        return tb_kernel_time(self.h, kind)

    def workspace_bytes(self):
        return tb_workspace_bytes(self.h)

    # -- helpers
    def _as_f64(self, a):
        import numpy as np
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            return a.to(dtype=self._torch.float64).contiguous()
        return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1, 3))

    def _as_f32(self, a):
        import numpy as np
        if hasattr(a, "data_ptr"):
            return a.to(dtype=self._torch.float32).contiguous()
        return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _autograd_function():
    import torch

    class _AcousticTraces(torch.autograd.Function):
        """traces = F(vp) through the C ABI; backward by tb_adjoint_gradient.

        The time step and the damping are held fixed (pass them explicitly),
        which is what the gradient differentiates."""

        @staticmethod
        def forward(ctx, vp, prop, src_xyz, wavelets, rec_xyz, nt, dt, damp, n_snapshots):
            prop.set_model(vp.detach(), damp=damp, dt=dt)
            prop.set_sources(src_xyz, wavelets)
            prop.set_receivers(rec_xyz)
            traces = prop.forward(nt, schedule="onestep")
            ctx.prop, ctx.nt, ctx.nsnap = prop, nt, n_snapshots
            ctx.vp_shape = vp.shape
            return traces

        @staticmethod
        def backward(ctx, grad_traces):
            g = torch.empty(ctx.vp_shape, dtype=torch.float32, device="cuda")
            ctx.prop.adjoint_gradient(ctx.nt, grad_traces.contiguous(), grad_vp=g, n_snapshots=ctx.nsnap)
            return g, None, None, None, None, None, None, None, None

    return _AcousticTraces


class AcousticTraces:
    """torch.autograd.Function-style entry: AcousticTraces.apply(vp, prop,
    src_xyz, wavelets, rec_xyz, nt, dt, damp, n_snapshots) -> traces [nt, nrec]
    with d(traces)/d(vp) through the library's adjoint."""
    _fn = None

    @classmethod
    def apply(cls, *args):
        if cls._fn is None:
            cls._fn = _autograd_function()
        return cls._fn.apply(*args)
