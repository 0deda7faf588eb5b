"""Python binding of the lbrmhd C ABI (include/lbrmhd.h).

Argument marshalling only: every step of the method runs in the CUDA library
liblbrmhd.so. There is no CPU fallback: if the library cannot be built or
loaded, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

OK = 0
ERR_BAD_ARG, ERR_OOM, ERR_CUDA, ERR_NONCONVERGED, ERR_NONFINITE, ERR_TIMEOUT, ERR_STATE = -1, -2, -3, -4, -5, -6, -7
PERIODIC, OPEN, DRIVEN = 0, 1, 2
FP64, FP32, FP16_DEV = 0, 1, 2
RECOVERY_PLAIN, RECOVERY_MLP, RECOVERY_COLD = 0, 1, 2
FLAG_NO_EM_COLLISION, FLAG_UNSHIFTED_POWER, FLAG_ONE_PASS_RECOVERY, FLAG_GAUSS_CHARGE = 1, 2, 4, 8
FLAG_TMA_TILES, FLAG_FIRST_ORDER_FLUX = 16, 32
MLP_NPARAM, MLP_NFEAT, MLP_ROW = 9924, 20, 24
SCHED_PER_RUN, SCHED_BATCH, SCHED_PERSISTENT = 0, 1, 2
NMOMENTS, NDIAG, NTABLE, NHIST = 16, 10, 311, 17
MOMENT_NAMES = ["n", "p", "eps", "ux", "uy", "uz", "Ex", "Ey", "Ez", "Bx", "By", "Bz", "rho_c", "Jx", "Jy", "Jz"]
DIAG_NAMES = ["N0", "T00", "T01", "T02", "T03", "rho_c", "divB_max", "divB_rms", "nonfinite", "cells"]

EXPORTED = [
    "lbrmhd_create", "lbrmhd_destroy", "lbrmhd_set_stream", "lbrmhd_init_fields", "lbrmhd_init_fields_device",
    "lbrmhd_step", "lbrmhd_get_moments", "lbrmhd_get_moments_device", "lbrmhd_get_populations",
    "lbrmhd_get_diagnostics", "lbrmhd_get_stats", "lbrmhd_state_bytes", "lbrmhd_get_state", "lbrmhd_set_state",
    "lbrmhd_run_cells", "lbrmhd_last_error", "lbrmhd_lattice_tables", "lbrmhd_get_diagnostics_noalloc",
    "lbrmhd_mlp_nparams", "lbrmhd_mlp_blob_bytes", "lbrmhd_mlp_pack", "lbrmhd_mlp_infer", "lbrmhd_mlp_grad",
    "lbrmhd_mlp_train", "lbrmhd_set_mlp_weights", "lbrmhd_set_mlp_samples", "lbrmhd_get_iteration_histogram",
    "lbrmhd_set_schedule", "lbrmhd_get_schedule", "lbrmhd_autotune", "lbrmhd_reconnection_rate",
    "lbrmhd_init_fields_relaxed", "lbrmhd_get_status", "lbrmhd_barrier_selftest",
]


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("bc", C.c_int32 * 6),
        ("tau", C.c_double), ("sigma", C.c_double), ("gamma_ad", C.c_double), ("alpha", C.c_double),
        ("c", C.c_double), ("dx", C.c_double), ("drive_u0", C.c_double),
        ("drive_layers", C.c_int32), ("precision", C.c_int32), ("recovery", C.c_int32), ("flags", C.c_int32),
        ("max_iters", C.c_int32), ("tol", C.c_double), ("drive_f0", C.c_double), ("drive_vmax", C.c_double),
    ]


class Schedule(C.Structure):
    _fields_ = [("kind", C.c_int32), ("bx", C.c_int32), ("waves", C.c_int32), ("order", C.c_int32),
                ("streams", C.c_int32), ("graph_steps", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def make_schedule(kind=SCHED_BATCH, bx=128, waves=0, order=0, streams=1, graph_steps=0) -> Schedule:
    return Schedule(int(kind), int(bx), int(waves), int(order), int(streams), int(graph_steps))


def make_params(nx, ny=1, nz=1, *, bc=(PERIODIC,) * 6, tau=1.0, sigma=100.0, gamma_ad=4.0 / 3.0, alpha=0.1, c=1.0,
                dx=1.0, drive_u0=0.0, drive_layers=0, precision=FP32, recovery=RECOVERY_PLAIN, flags=0, max_iters=0,
                tol=0.0, drive_f0=0.0, drive_vmax=0.0) -> Params:
    P = Params()
    P.nx, P.ny, P.nz = int(nx), int(ny), int(nz)
    for k in range(6):
        P.bc[k] = int(bc[k])
    P.tau, P.sigma, P.gamma_ad, P.alpha, P.c, P.dx = tau, sigma, gamma_ad, alpha, c, dx
    P.drive_u0, P.drive_layers = drive_u0, int(drive_layers)
    P.precision, P.recovery, P.flags, P.max_iters, P.tol = int(precision), int(recovery), int(flags), int(max_iters), tol
    P.drive_f0, P.drive_vmax = drive_f0, drive_vmax
    return P


_lock = threading.Lock()
_lib = None


class LbrmhdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lbrmhd error {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Loads liblbrmhd.so (building it with nvcc first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
        L = C.CDLL(path)
        vp, dp, i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int64
        L.lbrmhd_create.argtypes = [C.POINTER(Params), C.c_int, C.POINTER(C.c_void_p)]
        L.lbrmhd_destroy.argtypes = [vp]
        L.lbrmhd_set_stream.argtypes = [vp, vp]
        L.lbrmhd_init_fields.argtypes = [vp, C.c_int, dp, dp, dp, dp, dp]
        L.lbrmhd_init_fields_relaxed.argtypes = [vp, C.c_int, dp, dp, dp, dp, C.c_int, C.c_double,
                                                 C.POINTER(C.c_int), dp]
        L.lbrmhd_init_fields_device.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp]
        L.lbrmhd_step.argtypes = [vp, i64]
        L.lbrmhd_get_moments.argtypes = [vp, C.c_int, dp]
        L.lbrmhd_get_moments_device.argtypes = [vp, C.c_int, vp]
        L.lbrmhd_get_populations.argtypes = [vp, C.c_int, dp, dp, dp]
        L.lbrmhd_get_diagnostics.argtypes = [vp, C.c_int, dp]
        L.lbrmhd_get_diagnostics_noalloc.argtypes = [vp, C.c_int, vp]
        L.lbrmhd_get_stats.argtypes = [vp, C.c_int, C.POINTER(i64)]
        L.lbrmhd_get_status.argtypes = [vp, C.POINTER(i64)]
        L.lbrmhd_barrier_selftest.argtypes = [vp, C.c_int, C.c_double]
        L.lbrmhd_state_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.lbrmhd_get_state.argtypes = [vp, vp, C.c_size_t]
        L.lbrmhd_set_state.argtypes = [vp, vp, C.c_size_t]
        L.lbrmhd_run_cells.argtypes = [vp, C.c_int]
        L.lbrmhd_run_cells.restype = i64
        L.lbrmhd_last_error.argtypes = [vp]
        L.lbrmhd_last_error.restype = C.c_char_p
        L.lbrmhd_lattice_tables.argtypes = [dp, C.c_size_t]
        L.lbrmhd_mlp_nparams.argtypes = []
        L.lbrmhd_mlp_blob_bytes.argtypes = []
        L.lbrmhd_mlp_pack.argtypes = [vp, vp, vp]
        L.lbrmhd_mlp_infer.argtypes = [vp, vp, i64, vp, vp]
        L.lbrmhd_mlp_grad.argtypes = [vp, vp, i64, vp, vp]
        L.lbrmhd_mlp_train.argtypes = [vp, vp, vp, i64, C.c_int, C.c_int, C.c_float, C.c_uint64, vp, vp]
        L.lbrmhd_set_mlp_weights.argtypes = [vp, vp]
        L.lbrmhd_set_mlp_samples.argtypes = [vp, C.c_int, vp]
        L.lbrmhd_get_iteration_histogram.argtypes = [vp, C.c_int, C.POINTER(i64)]
        L.lbrmhd_set_schedule.argtypes = [vp, C.POINTER(Schedule)]
        L.lbrmhd_get_schedule.argtypes = [vp, C.POINTER(Schedule)]
        L.lbrmhd_autotune.argtypes = [vp, C.c_int, C.POINTER(Schedule), C.POINTER(C.c_double)]
        L.lbrmhd_reconnection_rate.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_double, dp]
        _lib = L
        return L


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, n) -> np.ndarray:
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(-1)
    if out.size != n:
        raise ValueError(f"expected {n} values, got {out.size}")
    return out


def lattice_tables() -> dict:
    """The lattice tables compiled into the library (needs no GPU)."""
    out = np.zeros(NTABLE)
    rc = load().lbrmhd_lattice_tables(_dp(out), NTABLE)
    if rc != OK:
        raise LbrmhdError(rc, "lattice_tables")
    o = 0

    def take(n, shape):
        nonlocal o
        v = out[o:o + n].reshape(shape)
        o += n
        return v

    return {"chat": take(57, (19, 3)), "w": take(19, (19,)), "wg": take(19, (19,)), "hop": take(72, (24, 3)),
            "e_over_c": take(72, (24, 3)), "b": take(72, (24, 3))}


def _ptr(t):
    """Device pointer of a torch tensor (contiguous) or an integer address."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("device arrays must be contiguous")
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(int(t))


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(getattr(stream, "cuda_stream", stream) or 0)


def _need_f32(t, n, what):
    import torch
    if t.dtype != torch.float32 or not t.is_cuda or t.numel() != n:
        raise ValueError(f"{what}: expected a cuda float32 tensor of {n} values")


def _rc(rc, what):
    if rc != OK:
        raise LbrmhdError(rc, what)


def mlp_pack(params, stream=None):
    """Packed inference blob (uint8 cuda tensor) of float32 parameters."""
    import torch
    _need_f32(params, MLP_NPARAM, "params")
    L = load()
    blob = torch.empty(L.lbrmhd_mlp_blob_bytes(), dtype=torch.uint8, device=params.device)
    _rc(L.lbrmhd_mlp_pack(_ptr(params), _ptr(blob), _stream_ptr(stream)), "mlp_pack")
    return blob


def mlp_infer(blob, features, stream=None):
    """Network outputs (n x 4) for feature rows (n x 20, cuda float32)."""
    import torch
    n = features.numel() // MLP_NFEAT
    _need_f32(features, n * MLP_NFEAT, "features")
    out = torch.empty((n, 4), dtype=torch.float32, device=features.device)
    _rc(load().lbrmhd_mlp_infer(_ptr(blob), _ptr(features), n, _ptr(out), _stream_ptr(stream)), "mlp_infer")
    return out


def mlp_grad(params, data, stream=None):
    """(loss, gradient) of the mean squared error over the sample rows (n x 24)."""
    import torch
    n = data.numel() // MLP_ROW
    _need_f32(params, MLP_NPARAM, "params")
    _need_f32(data, n * MLP_ROW, "data")
    g = torch.empty(MLP_NPARAM + 1, dtype=torch.float32, device=data.device)
    _rc(load().lbrmhd_mlp_grad(_ptr(params), _ptr(data), n, _ptr(g), _stream_ptr(stream)), "mlp_grad")
    return float(g[MLP_NPARAM]), g[:MLP_NPARAM]


def mlp_train(params, adam, data, steps, batch, lr, seed=1, stream=None):
    """Adam steps on mini-batches of the sample rows; updates params and adam
    (2 x MLP_NPARAM) in place and returns the per-step mini-batch losses."""
    import torch
    n = data.numel() // MLP_ROW
    _need_f32(params, MLP_NPARAM, "params")
    _need_f32(adam, 2 * MLP_NPARAM, "adam")
    _need_f32(data, n * MLP_ROW, "data")
    loss = torch.empty(max(int(steps), 1), dtype=torch.float32, device=data.device)
    _rc(load().lbrmhd_mlp_train(_ptr(params), _ptr(adam), _ptr(data), n, int(steps), int(batch), float(lr),
                                int(seed), _ptr(loss), _stream_ptr(stream)), "mlp_train")
    return loss[:int(steps)]


class Solver:
    """One handle of the library: n_runs independent runs advanced together."""

    def __init__(self, params, stream=None):
        L = load()
        plist = params if isinstance(params, (list, tuple)) else [params]
        arr = (Params * len(plist))(*plist)
        h = C.c_void_p()
        rc = L.lbrmhd_create(arr, len(plist), C.byref(h))
        if rc != OK:
            raise LbrmhdError(rc, L.lbrmhd_last_error(None).decode())
        self._L, self._h, self.params = L, h, list(plist)
        self.cells = [int(L.lbrmhd_run_cells(h, r)) for r in range(len(plist))]
        if stream is not None:
            self.set_stream(stream)

    def _check(self, rc):
        if rc != OK:
            raise LbrmhdError(rc, self._L.lbrmhd_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.lbrmhd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an integer cudaStream_t or None."""
        ptr = getattr(stream, "cuda_stream", stream)
        self._check(self._L.lbrmhd_set_stream(self._h, C.c_void_p(ptr or 0)))

    def init_fields(self, run, n, p, u, B, E=None):
        N = self.cells[run]
        n, p, u, B = _f64(n, N), _f64(p, N), _f64(u, 3 * N), _f64(B, 3 * N)
        Ep = None if E is None else _f64(E, 3 * N)
        self._check(self._L.lbrmhd_init_fields(self._h, run, _dp(n), _dp(p), _dp(u), _dp(B),
                                               None if Ep is None else _dp(Ep)))

    def init_fields_relaxed(self, run, n, p, u, B, max_iters=200, tol=1e-6):
        """Initial state whose E, J have relaxed with n, p, u, B held (the
        flare set-up's iterative initialisation); returns (steps, residual)."""
        N = self.cells[run]
        n, p, u, B = _f64(n, N), _f64(p, N), _f64(u, 3 * N), _f64(B, 3 * N)
        its, res = C.c_int(0), C.c_double(0.0)
        self._check(self._L.lbrmhd_init_fields_relaxed(self._h, run, _dp(n), _dp(p), _dp(u), _dp(B), int(max_iters),
                                                       float(tol), C.byref(its), C.byref(res)))
        return its.value, res.value

    def init_fields_device(self, run, n, p, u, B, E=None):
        """Device float64 arrays: torch tensors (contiguous, cuda) or integer pointers."""
        ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr() if hasattr(t, "data_ptr") else int(t))
        self._check(self._L.lbrmhd_init_fields_device(self._h, run, ptr(n), ptr(p), ptr(u), ptr(B), ptr(E)))

    def step(self, nsteps=1):
        self._check(self._L.lbrmhd_step(self._h, int(nsteps)))

    def moments(self, run=0) -> np.ndarray:
        out = np.zeros(NMOMENTS * self.cells[run])
        self._check(self._L.lbrmhd_get_moments(self._h, run, _dp(out)))
        return out.reshape(NMOMENTS, self.cells[run])

    def moments_device(self, run, out_ptr):
        ptr = out_ptr.data_ptr() if hasattr(out_ptr, "data_ptr") else int(out_ptr)
        self._check(self._L.lbrmhd_get_moments_device(self._h, run, C.c_void_p(ptr)))

    def populations(self, run=0):
        N = self.cells[run]
        f, g, h = np.zeros(19 * N), np.zeros(19 * N), np.zeros(25 * N)
        self._check(self._L.lbrmhd_get_populations(self._h, run, _dp(f), _dp(g), _dp(h)))
        return f.reshape(19, N), g.reshape(19, N), h.reshape(25, N)

    def diagnostics(self, run=0, check=True) -> np.ndarray:
        out = np.zeros(NDIAG)
        rc = self._L.lbrmhd_get_diagnostics(self._h, run, _dp(out))
        if check or rc not in (OK, ERR_NONFINITE):
            self._check(rc)
        return out

    def stats(self, run=0) -> dict:
        out = (C.c_int64 * 4)()
        self._check(self._L.lbrmhd_get_stats(self._h, run, out))
        return {"steps": out[0], "recover_fail": out[1], "iter_total": out[2], "iter_max": out[3]}

    def status(self) -> dict:
        """Health of the handle (synchronises): status bits of the step kernels,
        recovery failures over all runs, runs on the TMA tile kernel, and the
        call's return code (OK, ERR_NONCONVERGED or ERR_TIMEOUT)."""
        out = (C.c_int64 * 3)()
        rc = self._L.lbrmhd_get_status(self._h, out)
        if rc not in (OK, ERR_NONCONVERGED, ERR_TIMEOUT):
            self._check(rc)
        return {"bits": out[0], "recover_fail": out[1], "tiled_runs": out[2], "rc": rc}

    def iteration_histogram(self, run=0) -> np.ndarray:
        """Recovery iteration counts since init: [k] = cell updates converged in
        k + 1 iterations (last bin: NHIST or more)."""
        out = (C.c_int64 * NHIST)()
        self._check(self._L.lbrmhd_get_iteration_histogram(self._h, run, out))
        return np.array(out[:], dtype=np.int64)

    def reconnection_rate(self, run, y_lo, y_hi, B0) -> dict:
        """R = (E^z - E^z_0) / B0 at the null point of rows [y_lo, y_hi) (2-D runs)."""
        out = np.zeros(4)
        self._check(self._L.lbrmhd_reconnection_rate(self._h, run, int(y_lo), int(y_hi), float(B0), _dp(out)))
        return {"R": out[0], "x": int(out[1]) if np.isfinite(out[1]) else -1,
                "y": int(out[2]) if np.isfinite(out[2]) else -1, "B": out[3]}

    def get_state(self) -> bytes:
        n = C.c_size_t()
        self._check(self._L.lbrmhd_state_bytes(self._h, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(self._L.lbrmhd_get_state(self._h, buf, n.value))
        return buf.raw

    def set_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        self._check(self._L.lbrmhd_set_state(self._h, buf, len(blob)))

    def set_schedule(self, sched: Schedule | None = None, **kw):
        """Launch schedule (see lbrmhd_schedule); keyword arguments build one."""
        sched = sched if sched is not None else make_schedule(**kw)
        self._check(self._L.lbrmhd_set_schedule(self._h, C.byref(sched)))

    def schedule(self) -> Schedule:
        out = Schedule()
        self._check(self._L.lbrmhd_get_schedule(self._h, C.byref(out)))
        return out

    def autotune(self, trials=3):
        """Times the candidate schedules on dry steps, keeps the fastest;
        returns (schedule, ms per step)."""
        best, ms = Schedule(), C.c_double()
        self._check(self._L.lbrmhd_autotune(self._h, int(trials), C.byref(best), C.byref(ms)))
        return best, ms.value

    def set_mlp_weights(self, params):
        """Network of the learned recovery seed (cuda float32, MLP_NPARAM)."""
        _need_f32(params, MLP_NPARAM, "params")
        self._check(self._L.lbrmhd_set_mlp_weights(self._h, _ptr(params)))

    def set_mlp_samples(self, run, samples):
        """Attaches a cuda float32 buffer of cells x 24 that each following
        step fills with training samples (None detaches)."""
        if samples is not None:
            _need_f32(samples, self.cells[run] * MLP_ROW, "samples")
        self._check(self._L.lbrmhd_set_mlp_samples(self._h, run, _ptr(samples)))
        self._samples = samples  # keep the buffer alive while attached
