"""ctypes binding of ``libadorym.so`` (argument marshalling only).

Every step of the loss/gradient path runs in the library's CUDA kernels; this module only
converts Python/torch/numpy arguments to the C ABI declared in ``include/adorym.h``.  If the
library has not been built the import fails loudly: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libadorym.so")

OK, EINVAL, ENOMEM, ETIMEDOUT, EDEVICE, ENOENT, ETOOBIG, EDATA, ECANCELED = 0, 1, 2, 3, 4, 5, 6, 7, 8
NOALLOC_SCRATCH_BYTES = 64 << 20
LOSS = {"lsq": 0, "poisson": 1}

EXPORTS = ["adorym_create", "adorym_destroy", "adorym_last_error", "adorym_register_object",
           "adorym_unregister_object", "adorym_forward", "adorym_loss_grad", "adorym_submit", "adorym_poll",
           "adorym_serve_config", "adorym_serve_stats", "adorym_workspace_bytes", "adorym_enable_kernel_timing",
           "adorym_kernel_ms", "adorym_loss_grad_noalloc", "adorym_loss_grad_ext", "adorym_regularize",
           "adorym_l1_weights", "adorym_check", "adorym_kernel_launches",
           "adorym_fp32_peak", "adorym_cancel", "adorym_inject_alloc_failures", "adorym_set_wait_limits",
           "adorym_poll_times"]
WAIT_DEFAULT, WAIT_GIVE_UP = -1, -2


class Problem(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("L", ctypes.c_int), ("M", ctypes.c_int), ("B", ctypes.c_int),
                ("Ly", ctypes.c_int), ("Lx", ctypes.c_int), ("Lz", ctypes.c_int),
                ("kdz", ctypes.c_double), ("lambda_dz_over_px2", ctypes.c_double),
                ("farfield", ctypes.c_int), ("n_dist", ctypes.c_int), ("nf", ctypes.c_double * 4),
                ("loss", ctypes.c_int), ("eps", ctypes.c_double), ("tomo", ctypes.c_int),
                ("theta", ctypes.c_double), ("checkpoint_every", ctypes.c_int), ("gaps", ctypes.c_void_p)]

    @staticmethod
    def of(d: dict) -> "Problem":
        p = Problem()
        gaps = d.get("gaps")
        if gaps is not None:
            p._gaps = (ctypes.c_double * len(gaps))(*[float(v) for v in gaps])   # kept alive with p
            p.gaps = ctypes.cast(p._gaps, ctypes.c_void_p)
        for k in ("N", "L", "M", "B", "Ly", "Lx", "Lz"):
            setattr(p, k, int(d[k]))
        p.kdz = float(d["kdz"])
        p.lambda_dz_over_px2 = float(d.get("lambda_dz_over_px2", 0.0))
        p.farfield = int(d.get("farfield", 1))
        nf = list(d.get("nf", []))
        p.n_dist = len(nf)
        for i, v in enumerate(nf[:4]):
            p.nf[i] = float(v)
        loss = d.get("loss", "lsq")
        p.loss = LOSS[loss] if isinstance(loss, str) else int(loss)
        p.eps = float(d.get("eps", 1e-6))
        p.tomo = int(d.get("tomo", 0))
        p.theta = float(d.get("theta", 0.0))
        p.checkpoint_every = int(d.get("checkpoint_every", 0))
        return p


class Grads(ctypes.Structure):
    _fields_ = [("loss", ctypes.c_void_p), ("g_delta", ctypes.c_void_p), ("g_beta", ctypes.c_void_p),
                ("g_probe", ctypes.c_void_p), ("g_pos", ctypes.c_void_p), ("g_nf", ctypes.c_void_p),
                ("I_out", ctypes.c_void_p), ("g_gaps", ctypes.c_void_p), ("g_offset", ctypes.c_void_p)]


class Reg(ctypes.Structure):
    _fields_ = [("alpha_delta", ctypes.c_double), ("alpha_beta", ctypes.c_double), ("w_delta", ctypes.c_void_p),
                ("w_beta", ctypes.c_void_p), ("gamma_tv", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("problem", Problem), ("obj_id", ctypes.c_int),
                ("probe", ctypes.c_void_p), ("pos", ctypes.c_void_p), ("I_meas", ctypes.c_void_p),
                ("loss_out", ctypes.c_void_p), ("g_delta", ctypes.c_void_p), ("g_beta", ctypes.c_void_p),
                ("g_probe", ctypes.c_void_p), ("g_pos", ctypes.c_void_p), ("I_out", ctypes.c_void_p)]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2012_12686_gb300.build` "
                               "(the CUDA path has no fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64
        L.adorym_create.argtypes = [ctypes.POINTER(vp), i32, vp]
        L.adorym_destroy.argtypes = [vp]
        L.adorym_destroy.restype = None
        L.adorym_last_error.argtypes = [vp]
        L.adorym_last_error.restype = ctypes.c_char_p
        L.adorym_register_object.argtypes = [vp, vp, vp, i32, i32, i32, ctypes.POINTER(i32)]
        L.adorym_unregister_object.argtypes = [vp, i32]
        L.adorym_forward.argtypes = [vp, ctypes.POINTER(Problem), i32, vp, vp, vp]
        L.adorym_loss_grad.argtypes = [vp, ctypes.POINTER(Problem), i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.adorym_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(u64)]
        L.adorym_poll.argtypes = [vp, u64, ctypes.c_int64]
        L.adorym_poll_times.argtypes = [vp, u64, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]
        L.adorym_serve_config.argtypes = [vp, i32, u64]
        L.adorym_serve_stats.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.adorym_workspace_bytes.argtypes = [ctypes.POINTER(Problem), i32, ctypes.POINTER(u64)]
        L.adorym_enable_kernel_timing.argtypes = [vp, i32]
        L.adorym_kernel_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
        L.adorym_regularize.argtypes = [vp, i32, ctypes.POINTER(Reg), vp, vp, vp]
        L.adorym_l1_weights.argtypes = [vp, i32, ctypes.c_double, vp, vp]
        L.adorym_loss_grad_ext.argtypes = [vp, ctypes.POINTER(Problem), i32, vp, vp, vp, ctypes.POINTER(Grads)]
        L.adorym_loss_grad_noalloc.argtypes = [vp, ctypes.POINTER(Problem), vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                               vp]
        L.adorym_check.argtypes = [vp]
        L.adorym_kernel_launches.argtypes = []
        L.adorym_fp32_peak.argtypes = [i32, ctypes.POINTER(ctypes.c_double)]
        L.adorym_cancel.argtypes = [vp, u64]
        L.adorym_inject_alloc_failures.argtypes = [vp, i32]
        L.adorym_set_wait_limits.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
        for name in EXPORTS:
            if name not in ("adorym_destroy", "adorym_last_error", "adorym_kernel_launches"):
                getattr(L, name).restype = ctypes.c_int
        L.adorym_kernel_launches.restype = ctypes.c_uint64
        _lib = L
    return _lib


def fp32_peak(device: int = 0) -> float:
    """Measured FP32 FMA throughput of the device, TFLOP/s."""
    v = ctypes.c_double()
    rc = lib().adorym_fp32_peak(device, ctypes.byref(v))
    if rc:
        raise AdorymError(rc, "fp32 peak measurement failed")
    return v.value


def kernel_launches() -> int:
    """Kernels this library has launched in the process so far (differences give a region's count)."""
    return int(lib().adorym_kernel_launches())


def _ptr(x):
    """Address of a torch tensor / numpy array (must be contiguous), an int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported argument type {type(x)}")


class AdorymError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"adorym error {code}: {msg}")
        self.code = code


class Engine:
    """One library context bound to a CUDA device and stream (default: torch's current stream)."""

    def __init__(self, device: int = 0, stream: int | None = None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        self._ctx = ctypes.c_void_p()
        rc = lib().adorym_create(ctypes.byref(self._ctx), device, ctypes.c_void_p(stream))
        if rc:
            raise AdorymError(rc, "adorym_create failed")

    def close(self):
        if self._ctx:
            lib().adorym_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return lib().adorym_last_error(self._ctx).decode()

    def _check(self, rc):
        if rc:
            raise AdorymError(rc, self.last_error())
        return rc

    def register_object(self, delta, beta) -> int:
        Lz, Ly, Lx = delta.shape
        oid = ctypes.c_int()
        self._check(lib().adorym_register_object(self._ctx, _ptr(delta), _ptr(beta), Lz, Ly, Lx, ctypes.byref(oid)))
        return oid.value

    def unregister_object(self, obj_id: int):
        self._check(lib().adorym_unregister_object(self._ctx, obj_id))

    def forward(self, problem, obj_id, probe, pos, I_out):
        p = problem if isinstance(problem, Problem) else Problem.of(problem)
        return self._check(lib().adorym_forward(self._ctx, ctypes.byref(p), obj_id, _ptr(probe), _ptr(pos),
                                                _ptr(I_out)))

    def loss_grad(self, problem, obj_id, probe, pos, I_meas, loss_out=None, g_delta=None, g_beta=None,
                  g_probe=None, g_pos=None, I_out=None):
        p = problem if isinstance(problem, Problem) else Problem.of(problem)
        return self._check(lib().adorym_loss_grad(self._ctx, ctypes.byref(p), obj_id, _ptr(probe), _ptr(pos),
                                                  _ptr(I_meas), _ptr(loss_out), _ptr(g_delta), _ptr(g_beta),
                                                  _ptr(g_probe), _ptr(g_pos), _ptr(I_out)))

    def loss_grad_ext(self, problem, obj_id, probe, pos, I_meas, loss_out=None, g_delta=None, g_beta=None,
                      g_probe=None, g_pos=None, g_nf=None, I_out=None, g_gaps=None, g_offset=None):
        """adorym_loss_grad_ext: as loss_grad, plus g_nf (near field: dL/dN_F per problem and distance),
        g_gaps (variable slice spacing: dL/d(lambda dz_j / dx^2)) and g_offset (far field: [2] gradient
        w.r.t. one position offset shared by the whole batch, the per-angle offset)."""
        p = problem if isinstance(problem, Problem) else Problem.of(problem)
        g = Grads()
        for k, v in (("loss", loss_out), ("g_delta", g_delta), ("g_beta", g_beta), ("g_probe", g_probe),
                     ("g_pos", g_pos), ("g_nf", g_nf), ("I_out", I_out), ("g_gaps", g_gaps),
                     ("g_offset", g_offset)):
            setattr(g, k, _ptr(v))
        return self._check(lib().adorym_loss_grad_ext(self._ctx, ctypes.byref(p), obj_id, _ptr(probe), _ptr(pos),
                                                      _ptr(I_meas), ctypes.byref(g)))

    def regularize(self, obj_id, alpha_delta=0.0, alpha_beta=0.0, gamma_tv=0.0, w_delta=None, w_beta=None,
                   loss_out=None, g_delta=None, g_beta=None):
        """adorym_regularize: l1 / reweighted l1 / TV regularizer value and gradient (Eq. tikhonov)."""
        r = Reg(float(alpha_delta), float(alpha_beta), _ptr(w_delta), _ptr(w_beta), float(gamma_tv))
        return self._check(lib().adorym_regularize(self._ctx, obj_id, ctypes.byref(r), _ptr(loss_out), _ptr(g_delta),
                                                   _ptr(g_beta)))

    def l1_weights(self, obj_id, eps, w_delta, w_beta):
        return self._check(lib().adorym_l1_weights(self._ctx, obj_id, float(eps), _ptr(w_delta), _ptr(w_beta)))

    def enable_kernel_timing(self, on: bool = True):
        self._check(lib().adorym_enable_kernel_timing(self._ctx, 1 if on else 0))

    def kernel_ms(self) -> float:
        v = ctypes.c_float()
        self._check(lib().adorym_kernel_ms(self._ctx, ctypes.byref(v)))
        return v.value

    # ---- serving
    def serve_config(self, slots: int, budget_bytes: int = 0):
        self._check(lib().adorym_serve_config(self._ctx, slots, budget_bytes))

    def submit(self, problem, obj_id, probe, pos, I_meas, loss_out=None, g_delta=None, g_beta=None,
               g_probe=None, g_pos=None, I_out=None) -> int:
        r = Request()
        r.problem = problem if isinstance(problem, Problem) else Problem.of(problem)
        r.obj_id = obj_id
        for k, v in (("probe", probe), ("pos", pos), ("I_meas", I_meas), ("loss_out", loss_out),
                     ("g_delta", g_delta), ("g_beta", g_beta), ("g_probe", g_probe), ("g_pos", g_pos),
                     ("I_out", I_out)):
            setattr(r, k, _ptr(v))
        t = ctypes.c_uint64()
        self._check(lib().adorym_submit(self._ctx, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int, timeout_us: int = -1) -> int:
        rc = lib().adorym_poll(self._ctx, ticket, timeout_us)
        if rc not in (OK, ETIMEDOUT):
            raise AdorymError(rc, self.last_error())
        return rc

    def poll_times(self, ticket: int, timeout_us: int = -1):
        """adorym_poll_times: (rc, queued_us, run_us, admitted_at_us) -- time waiting for admission,
        time from admission to completion, and the admission instant (host clock); rc is OK or
        ETIMEDOUT, other codes raise."""
        t = (ctypes.c_double * 3)()
        rc = lib().adorym_poll_times(self._ctx, ticket, timeout_us, t)
        if rc not in (OK, ETIMEDOUT):
            raise AdorymError(rc, self.last_error())
        return rc, t[0], t[1], t[2]

    def check(self) -> int:
        """Wait for the context's stream and raise on the last call's device status word (EDATA:
        invalid positions / shifts found by the kernels)."""
        return self._check(lib().adorym_check(self._ctx))

    def cancel(self, ticket: int) -> int:
        """Cancel a request still waiting for admission (its poll then reports ECANCELED)."""
        return self._check(lib().adorym_cancel(self._ctx, ticket))

    def inject_alloc_failures(self, count: int) -> int:
        """Make the next `count` workspace allocations fail with ENOMEM (host side; for tests)."""
        return self._check(lib().adorym_inject_alloc_failures(self._ctx, count))

    def serve_stats(self):
        c, w = ctypes.c_uint64(), ctypes.c_uint64()
        self._check(lib().adorym_serve_stats(self._ctx, ctypes.byref(c), ctypes.byref(w)))
        return c.value, w.value


def loss_grad_noalloc(stream, problem, delta, beta, probe, pos, I_meas, loss_out=None, g_delta=None, g_beta=None,
                      g_probe=None, g_pos=None, I_out=None, status=None) -> int:
    """adorym_loss_grad_noalloc: same computation as Engine.loss_grad with no device allocation
    (fixed 64 MiB scratch); all arrays must be device memory.  `status`: optional device int32
    tensor, zeroed by the caller, into which the kernels OR the call's status bits.  Returns the
    library's code."""
    p = problem if isinstance(problem, Problem) else Problem.of(problem)
    return lib().adorym_loss_grad_noalloc(ctypes.c_void_p(stream), ctypes.byref(p), _ptr(delta), _ptr(beta),
                                          _ptr(probe), _ptr(pos), _ptr(I_meas), _ptr(loss_out), _ptr(g_delta),
                                          _ptr(g_beta), _ptr(g_probe), _ptr(g_pos), _ptr(I_out), _ptr(status))


def set_wait_limits(segment_cycles=WAIT_DEFAULT, checkpoint_cycles=WAIT_DEFAULT, tile_copy_cycles=WAIT_DEFAULT):
    """adorym_set_wait_limits: cycle limits of the bounded device-side waits (test hook; the
    defaults are restored by WAIT_DEFAULT).  Returns the library's code."""
    return lib().adorym_set_wait_limits(int(segment_cycles), int(checkpoint_cycles), int(tile_copy_cycles))


def workspace_bytes(problem, grads: int = 7) -> int:
    p = problem if isinstance(problem, Problem) else Problem.of(problem)
    out = ctypes.c_uint64()
    rc = lib().adorym_workspace_bytes(ctypes.byref(p), grads, ctypes.byref(out))
    if rc:
        raise AdorymError(rc, "invalid problem")
    return out.value
