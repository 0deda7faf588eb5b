"""ctypes binding of the FP64 C oracle (``lbrmhd_oracle.c``).

TEST INFRASTRUCTURE ONLY. Argument marshalling for the plain C restatement of
arXiv:1508.03452; every equation lives in the C file, next to its citation.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbrmhd_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liblbrmhd_oracle.so")

PERIODIC, OPEN, DRIVEN = 0, 1, 2
NO_EM_COLLISION, FIRST_ORDER, IMPLICIT_AS_PRINTED, PRINTED_FEQ, ONE_PASS_RECOVERY, GAUSS_CHARGE = 1, 2, 4, 8, 16, 32
# primitive layout (per cell)
N_, EPS_, U_, E_, B_, RHOC_, J_, NPRIM = 0, 1, 2, 5, 8, 11, 12, 15
# get_moments output rows
OUT_FIELDS = ["n", "p", "eps", "ux", "uy", "uz", "Ex", "Ey", "Ez", "Bx", "By", "Bz", "rho_c", "Jx", "Jy", "Jz"]


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("bc", C.c_int32 * 6),
        ("tau", C.c_double), ("sigma", C.c_double), ("gamma_ad", C.c_double),
        ("alpha", C.c_double), ("c", C.c_double), ("dx", C.c_double), ("nu", C.c_double),
        ("drive_u0", C.c_double), ("drive_layers", C.c_int32), ("flags", C.c_int32),
        ("threads", C.c_int32), ("max_power_iters", C.c_int32), ("power_tol", C.c_double),
        ("drive_f0", C.c_double), ("drive_vmax", C.c_double),
    ]


class Lattice(C.Structure):
    _fields_ = [
        ("nu", C.c_double), ("ca", C.c_double), ("ct_c0", C.c_double), ("c0", C.c_double), ("ct", C.c_double),
        ("w", C.c_double * 19), ("wg", C.c_double * 19), ("p", (C.c_double * 4) * 19),
        ("chat", (C.c_int * 3) * 19),
        ("v", (C.c_double * 3) * 24), ("e", (C.c_double * 3) * 24), ("b", (C.c_double * 3) * 24),
        ("hop", (C.c_int * 3) * 24),
    ]


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available) into oracle/_build."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "lbrmhd_oracle.h"))
    ):
        return LIB_PATH
    base = ["gcc", "-std=c11", "-D_DEFAULT_SOURCE", "-O2", "-fPIC", "-shared", "-o", LIB_PATH + ".tmp", SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(LIB_PATH + ".tmp", LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            P = C.POINTER(Params)
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [P]
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_init.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
            L.orc_step.argtypes = [C.c_void_p, C.c_int64]
            L.orc_get_moments.argtypes = [C.c_void_p, dp]
            L.orc_get_state.argtypes = [C.c_void_p, dp, dp, dp, dp]
            L.orc_set_state.argtypes = [C.c_void_p, dp, dp, dp, dp]
            L.orc_update_cells.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.c_int64, dp, dp, dp, dp]
            L.orc_stats.argtypes = [C.c_void_p, C.POINTER(C.c_int64)]
            L.orc_get_post_collision.argtypes = [C.c_void_p, dp, dp, dp]
            L.orc_update_cells_from.argtypes = [C.c_void_p, dp, dp, dp, dp, C.POINTER(C.c_int64), C.c_int64,
                                                dp, dp, dp, dp]
            L.orc_get_lattice.argtypes = [P, C.POINTER(Lattice)]
            L.orc_dt.restype = C.c_double
            L.orc_dt.argtypes = [P]
            L.orc_courant.restype = C.c_double
            L.orc_courant.argtypes = [P, C.POINTER(Lattice)]
            L.orc_feq.argtypes = [P, C.POINTER(Lattice), C.c_double, C.c_double, dp, dp, dp, dp]
            L.orc_geq.argtypes = [P, C.POINTER(Lattice), C.c_double, dp, dp]
            L.orc_heq.argtypes = [P, C.POINTER(Lattice), dp, dp, dp, C.c_double, dp]
            L.orc_ohm_current.argtypes = [P, dp, dp, dp, C.c_double, dp]
            L.orc_ohm_solve.argtypes = [P, dp, dp, dp, C.c_double, dp]
            L.orc_moments.argtypes = [C.POINTER(Lattice), dp, dp, dp, dp, dp, dp, dp, dp]
            L.orc_maxwell_tensor.argtypes = [C.c_double, dp, dp, dp]
            L.orc_em_ff.argtypes = [P, dp, dp, dp]
            L.orc_landau.restype = C.c_int
            L.orc_landau.argtypes = [P, dp, dp, dp, dp, dp, dp]
            L.orc_recover_cell.restype = C.c_int
            L.orc_recover_cell.argtypes = [P, C.POINTER(Lattice), dp, dp, dp, dp, dp]
            L.orc_stream_population.argtypes = [P, C.c_int, dp, dp]
            L.orc_drive_velocity.argtypes = [P, C.c_int, C.c_int, dp]
            L.orc_drive_force.argtypes = [P, C.c_int, C.c_int, dp]
            L.orc_force_populations.argtypes = [P, C.POINTER(Lattice), dp, dp, dp]
            L.orc_force_on.restype = C.c_int
            L.orc_force_on.argtypes = [C.c_void_p]
            L.orc_init_relaxed.restype = C.c_int
            L.orc_init_relaxed.argtypes = [C.c_void_p, dp, dp, dp, dp, C.c_int, C.c_double, dp]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def make_params(nx=1, ny=1, nz=1, *, bc=(PERIODIC,) * 6, tau=1.0, sigma=100.0, gamma_ad=4.0 / 3.0, alpha=0.1,
                c=1.0, dx=1.0, nu=0.0, drive_u0=0.0, drive_layers=0, flags=0, threads=1,
                max_power_iters=1000, power_tol=1e-14, drive_f0=0.0, drive_vmax=0.0) -> Params:
    P = Params()
    P.nx, P.ny, P.nz = nx, ny, nz
    for k in range(6):
        P.bc[k] = int(bc[k])
    P.tau, P.sigma, P.gamma_ad, P.alpha, P.c, P.dx, P.nu = tau, sigma, gamma_ad, alpha, c, dx, nu
    P.drive_u0, P.drive_layers, P.flags, P.threads = drive_u0, drive_layers, flags, threads
    P.max_power_iters, P.power_tol = max_power_iters, power_tol
    P.drive_f0, P.drive_vmax = drive_f0, drive_vmax
    return P


def lattice(P: Params) -> dict:
    L = Lattice()
    lib().orc_get_lattice(C.byref(P), C.byref(L))
    return {
        "nu": L.nu, "ca": L.ca, "ct_c0": L.ct_c0, "c0": L.c0, "ct": L.ct,
        "w": np.array(L.w[:]), "wg": np.array(L.wg[:]),
        "p": np.array([list(r) for r in L.p]), "chat": np.array([list(r) for r in L.chat]),
        "v": np.array([list(r) for r in L.v]), "e": np.array([list(r) for r in L.e]),
        "b": np.array([list(r) for r in L.b]), "hop": np.array([list(r) for r in L.hop]),
        "_struct": L,
    }


def dt(P: Params) -> float:
    return lib().orc_dt(C.byref(P))


def courant(P: Params) -> float:
    L = Lattice()
    lib().orc_get_lattice(C.byref(P), C.byref(L))
    return lib().orc_courant(C.byref(P), C.byref(L))


def _lat(P):
    L = Lattice()
    lib().orc_get_lattice(C.byref(P), C.byref(L))
    return L


def feq(P, n, eps, u, E, B) -> np.ndarray:
    out = np.zeros(19)
    u, E, B = _f64(u), _f64(E), _f64(B)
    lib().orc_feq(C.byref(P), C.byref(_lat(P)), float(n), float(eps), _dp(u), _dp(E), _dp(B), _dp(out))
    return out


def geq(P, n, u) -> np.ndarray:
    out = np.zeros(19)
    u = _f64(u)
    lib().orc_geq(C.byref(P), C.byref(_lat(P)), float(n), _dp(u), _dp(out))
    return out


def heq(P, E, B, J, rho_c) -> np.ndarray:
    out = np.zeros(25)
    E, B, J = _f64(E), _f64(B), _f64(J)
    lib().orc_heq(C.byref(P), C.byref(_lat(P)), _dp(E), _dp(B), _dp(J), float(rho_c), _dp(out))
    return out


def ohm_current(P, E, u, B, rho_c) -> np.ndarray:
    out = np.zeros(3)
    E, u, B = _f64(E), _f64(u), _f64(B)
    lib().orc_ohm_current(C.byref(P), _dp(E), _dp(u), _dp(B), float(rho_c), _dp(out))
    return out


def ohm_solve(P, Ep, u, B, rho_c) -> np.ndarray:
    out = np.zeros(3)
    Ep, u, B = _f64(Ep), _f64(u), _f64(B)
    lib().orc_ohm_solve(C.byref(P), _dp(Ep), _dp(u), _dp(B), float(rho_c), _dp(out))
    return out


def moments(P, f, g, h):
    f, g, h = _f64(f), _f64(g), _f64(h)
    T = np.zeros(16); N = np.zeros(4); Ep = np.zeros(3); B = np.zeros(3); rc = np.zeros(1)
    lib().orc_moments(C.byref(_lat(P)), _dp(f), _dp(g), _dp(h), _dp(T), _dp(N), _dp(Ep), _dp(B), _dp(rc))
    return T.reshape(4, 4), N, Ep, B, float(rc[0])


def em_ff(P, E, B) -> np.ndarray:
    out = np.zeros(16)
    E, B = _f64(E), _f64(B)
    lib().orc_em_ff(C.byref(P), _dp(E), _dp(B), _dp(out))
    return out.reshape(4, 4)


def landau(P, T, E_prev, B_prev, U_seed):
    T, E_prev, B_prev, U_seed = _f64(T).reshape(16), _f64(E_prev), _f64(B_prev), _f64(U_seed)
    U = np.zeros(4); lam = np.zeros(1)
    it = lib().orc_landau(C.byref(P), _dp(T), _dp(E_prev), _dp(B_prev), _dp(U_seed), _dp(U), _dp(lam))
    return it, U, float(lam[0])


def recover_cell(P, f, g, h, prim_prev):
    f, g, h, prim_prev = _f64(f), _f64(g), _f64(h), _f64(prim_prev)
    out = np.zeros(NPRIM)
    it = lib().orc_recover_cell(C.byref(P), C.byref(_lat(P)), _dp(f), _dp(g), _dp(h), _dp(prim_prev), _dp(out))
    return it, out


def stream_population(P, i, fi) -> np.ndarray:
    fi = _f64(fi).reshape(-1)
    out = np.zeros_like(fi)
    lib().orc_stream_population(C.byref(P), int(i), _dp(fi), _dp(out))
    return out


def drive_velocity(P, x, y) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_drive_velocity(C.byref(P), int(x), int(y), _dp(out))
    return out


def drive_force(P, x, y) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_drive_force(C.byref(P), int(x), int(y), _dp(out))
    return out


def force_populations(P, F, u) -> np.ndarray:
    """R25: the change of a cell's 19 streamed f under force density F for one
    step (u: the previous step's velocity)."""
    F, u = _f64(F).reshape(3), _f64(u).reshape(3)
    out = np.zeros(19)
    lib().orc_force_populations(C.byref(P), C.byref(_lat(P)), _dp(F), _dp(u), _dp(out))
    return out


class Sim:
    """Owning wrapper of one oracle simulation (arrays x-fastest, field-major)."""

    def __init__(self, P: Params):
        self.P = P
        self.N = P.nx * P.ny * P.nz
        self._h = lib().orc_create(C.byref(P))
        if not self._h:
            raise ValueError("oracle rejected the parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def init(self, n, p, u, B, E=None):
        N = self.N
        n = _f64(n).reshape(N); p = _f64(p).reshape(N)
        u = _f64(u).reshape(3 * N); B = _f64(B).reshape(3 * N)
        Ep = None if E is None else _f64(E).reshape(3 * N)
        rc = lib().orc_init(self._h, _dp(n), _dp(p), _dp(u), _dp(B), None if Ep is None else _dp(Ep))
        if rc != 0:
            raise ValueError("oracle init failed (superluminal velocity?)")

    def init_relaxed(self, n, p, u, B, max_iters=200, tol=1e-12):
        """R27: initial state with E (rho_c, J) relaxed under the scheme at
        fixed n, p, u, B; returns (steps taken, final residual)."""
        N = self.N
        n = _f64(n).reshape(N); p = _f64(p).reshape(N)
        u = _f64(u).reshape(3 * N); B = _f64(B).reshape(3 * N)
        res = C.c_double(0.0)
        k = lib().orc_init_relaxed(self._h, _dp(n), _dp(p), _dp(u), _dp(B), int(max_iters), float(tol),
                                   C.byref(res))
        if k < 0:
            raise ValueError("oracle init failed (superluminal velocity?)")
        return k, res.value

    def force_on(self) -> bool:
        """R26: whether the body force acts in the next step."""
        return bool(lib().orc_force_on(self._h))

    def step(self, nsteps: int) -> int:
        return lib().orc_step(self._h, int(nsteps))

    def moments(self) -> np.ndarray:
        out = np.zeros(16 * self.N)
        lib().orc_get_moments(self._h, _dp(out))
        return out.reshape(16, self.N)

    def state(self):
        N = self.N
        f = np.zeros(19 * N); g = np.zeros(19 * N); h = np.zeros(25 * N); pr = np.zeros(NPRIM * N)
        lib().orc_get_state(self._h, _dp(f), _dp(g), _dp(h), _dp(pr))
        return f.reshape(19, N), g.reshape(19, N), h.reshape(25, N), pr.reshape(NPRIM, N)

    def set_state(self, f, g, h, prim):
        f, g, h, prim = (_f64(a).reshape(-1) for a in (f, g, h, prim))
        lib().orc_set_state(self._h, _dp(f), _dp(g), _dp(h), _dp(prim))

    def post_collision(self):
        N = self.N
        f = np.zeros(19 * N); g = np.zeros(19 * N); h = np.zeros(25 * N)
        lib().orc_get_post_collision(self._h, _dp(f), _dp(g), _dp(h))
        return f.reshape(19, N), g.reshape(19, N), h.reshape(25, N)

    def update_cells(self, cells):
        cells = np.ascontiguousarray(np.asarray(cells, dtype=np.int64))
        m = len(cells)
        f = np.zeros(19 * m); g = np.zeros(19 * m); h = np.zeros(25 * m); pr = np.zeros(NPRIM * m)
        rc = lib().orc_update_cells(self._h, cells.ctypes.data_as(C.POINTER(C.c_int64)), m,
                                    _dp(f), _dp(g), _dp(h), _dp(pr))
        if rc != 0:
            raise RuntimeError(f"oracle update_cells failed ({rc})")
        return f.reshape(m, 19), g.reshape(m, 19), h.reshape(m, 25), pr.reshape(m, NPRIM)

    def update_cells_from(self, fc, gc, hc, prim, cells):
        """Streams and recovers the listed cells from given post-collision
        populations and primitives (ORC prim layout, NPRIM planes)."""
        fc, gc, hc, prim = (_f64(a).reshape(-1) for a in (fc, gc, hc, prim))
        cells = np.ascontiguousarray(np.asarray(cells, dtype=np.int64))
        m = len(cells)
        f = np.zeros(19 * m); g = np.zeros(19 * m); h = np.zeros(25 * m); pr = np.zeros(NPRIM * m)
        rc = lib().orc_update_cells_from(self._h, _dp(fc), _dp(gc), _dp(hc), _dp(prim),
                                         cells.ctypes.data_as(C.POINTER(C.c_int64)), m, _dp(f), _dp(g), _dp(h),
                                         _dp(pr))
        if rc != 0:
            raise RuntimeError(f"oracle update_cells_from failed ({rc})")
        return f.reshape(m, 19), g.reshape(m, 19), h.reshape(m, 25), pr.reshape(m, NPRIM)

    def stats(self):
        out = (C.c_int64 * 4)()
        lib().orc_stats(self._h, out)
        return {"steps": out[0], "iter_total": out[1], "iter_max": out[2], "recover_fail": out[3]}
