"""GPU parity: the CUDA library, called through its C ABI, against the FP64
CPU oracle on the same seeded inputs.

Bars: relative L2 per field group <= 1e-10 for the float64 build and <= 1e-5
for the float32 build after the stated step counts. Float32 meets 1e-5 on every
group of the Alfven wave (config 1, 500 steps) and on n, p, eps and B
everywhere. Three small-signal groups miss it, and are kept as strict expected
failures with their measured errors rather than a looser bar:
  * the reduced current sheet (config 2, 2000 steps): u 5.7e-5, E 1.5e-5. The
    flow there is ~2e-4 c, driven by the sheets' magnetic pressure, which the
    fluid populations carry as deviations of ~1e-2 of their scale; float32
    arithmetic on them adds ~3e-8 relative error to u per step (linear
    growth: 2.3e-6 at 60 steps, 1.05e-5 at 500, 4.3e-5 at 1000). Measured:
    neither storing the populations in float64 (the arithmetic is float32),
    nor a float64-level recovery stopping floor, nor a 10x tighter recovery
    tolerance, nor the Gauss-law charge changes it (all within 10 %). With
    float64 arithmetic on the same float32-stored populations u and E fall to
    6.5e-6 and 4.4e-6: the error is the float32 arithmetic, spread over the
    streaming, moment and collision stages (each alone in float64 removes
    7-28 % of it); the recovery in float64 changes nothing (6.0e-5).
  * the Kelvin-Helmholtz layers (config 3 form, 40 steps): E 3.7e-5, which is
    E_z = u_y B_x of the 1e-3 noise velocity u_y, resolved by float32 to
    ~1e-4 of itself (u as a group, dominated by the 0.2c shear, is 3.4e-6; a
    10x tighter recovery tolerance leaves E at 3.9e-5, float64 arithmetic on
    the float32-stored populations at 2.8e-5).
  * the 3-D periodic state (10 steps): rho_c 2.4e-5, the charge h_0 + sum h,
    a near-cancelling sum of the Maxwell populations (every other group is
    within 9.2e-7).
The float16-deviation build has no bar (its error is reported by the
benchmark) beyond a sanity bound. Integer-like checks (the EM permutation)
are bit-exact.
"""
import functools
import numpy as np
import pytest

import oracle as O
from paper_1508_03452_gb300 import lbrmhd as L
from paper_1508_03452_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GROUPS = {"n": (0,), "p": (1,), "eps": (2,), "u": (3, 4, 5), "E": (6, 7, 8), "B": (9, 10, 11), "rho_c": (12,)}
TOL = {L.FP64: 1e-10, L.FP32: 1e-5}
BC_ORC = {L.PERIODIC: O.PERIODIC, L.OPEN: O.OPEN, L.DRIVEN: O.DRIVEN}


ZERO = 1e-12  # a field whose oracle values all stay below this is physically zero


def rel_errors(mg, mo):
    """Relative L2 error per field group. A group the oracle keeps at round-off
    (e.g. rho_c when div E = 0, as in the 1-D and in-plane 2-D problems) has no
    meaningful relative error and is left out (name -> None)."""
    out = {}
    for name, rows in GROUPS.items():
        a, b = mg[list(rows)], mo[list(rows)]
        out[name] = None if np.abs(b).max() < ZERO else np.linalg.norm(a - b) / np.linalg.norm(b)
    return out


def run_pair(F, steps, precision, *, bc=(L.PERIODIC,) * 6, check_groups=None, **kw):
    okw = {k: v for k, v in kw.items() if k in ("sigma", "tau", "alpha", "c", "dx", "drive_u0", "drive_layers")}
    ref = O.Sim(O.make_params(F.nx, F.ny, F.nz, bc=tuple(BC_ORC[b] for b in bc), threads=8, **okw))
    ref.init(F.n, F.p, F.u, F.B, F.E)
    ref.step(steps)
    s = L.Solver(L.make_params(F.nx, F.ny, F.nz, bc=bc, precision=precision, **kw))
    s.init_fields(0, F.n, F.p, F.u, F.B, F.E)
    s.step(steps)
    errs = rel_errors(s.moments(), ref.moments())
    st = s.stats()
    s.close()
    assert st["recover_fail"] == 0, st
    return errs, ref


def assert_parity(errs, tol, skip=(), loose=None):
    """Every group within tol; groups in `loose` (name -> bar) within their own bar."""
    loose = loose or {}
    bad = {k: v for k, v in errs.items() if v is not None and k not in skip and not v <= loose.get(k, tol)}
    assert not bad, (bad, errs)


# float32 small-signal groups below 1e-5 only over shorter horizons (module docstring)
FP32_SMALL_SIGNAL = {"sheet": ("u", "E"), "kh": ("E",), "3d": ("rho_c",)}


@pytest.mark.parametrize("precision", [L.FP64, L.FP32])
def test_alfven_config1(precision):
    """Config 1 in full: 64 x 64 periodic Alfven wave, sigma = 1e6, 500 steps,
    every group within the bar (float32: u 3.9e-6, E 3.9e-6)."""
    F = W.alfven_wave(64, 64, 1)
    errs, _ = run_pair(F, 500, precision, sigma=1e6)
    assert_parity(errs, TOL[precision])


@pytest.mark.parametrize("case", ["alfven", "sheet"])
def test_fp32_all_groups_short_horizon(case):
    """float32 within 1e-5 on every field group over 60 steps (u and E reach
    ~1e-5 after ~100 steps; see the module docstring)."""
    F = W.alfven_wave(64, 16, 1) if case == "alfven" else W.current_sheet(160, 12, 1, delta=8.0)
    errs, _ = run_pair(F, 60, L.FP32, sigma=1e6 if case == "alfven" else 100.0)
    assert_parity(errs, 1e-5)


def _three_dimensional_state():
    rng = np.random.default_rng(70)
    nx, ny, nz = 24, 20, 18
    N = nx * ny * nz
    z, y, x = (a.reshape(-1) for a in np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij"))
    u = np.zeros((3, N))
    u[0] = 0.05 * np.sin(2 * np.pi * y / ny)
    u[1] = 0.03 * np.sin(2 * np.pi * z / nz)
    u[2] = 0.04 * np.cos(2 * np.pi * x / nx)
    B = np.zeros((3, N))  # divergence-free: each component varies across its own axis only
    B[0] = 0.1 + 0.02 * np.sin(2 * np.pi * z / nz)
    B[1] = 0.02 * np.sin(2 * np.pi * x / nx)
    B[2] = 0.05 + 0.02 * np.cos(2 * np.pi * y / ny)
    return W.Fields(nx, ny, nz, 1.0 + 0.05 * rng.uniform(size=N), np.ones(N), u, B)


@functools.lru_cache(maxsize=None)
def _case_errors(case, precision):
    if case == "sheet":
        F = W.current_sheet(160, 12, 1, delta=8.0)
        errs, _ = run_pair(F, 2000, precision, sigma=100.0)
    elif case == "3d":
        errs, _ = run_pair(_three_dimensional_state(), 10, precision, sigma=50.0)
    else:
        F = W.kelvin_helmholtz(136, 72, 1, V=0.2, ratio=10.0, B0=0.1, a=2.0, noise=1e-3, seed=3)
        errs, _ = run_pair(F, 40, precision, sigma=1e3)
    return errs


@pytest.mark.parametrize("precision", [L.FP64, L.FP32])
def test_current_sheet_reduced(precision):
    """Config 2 on a reduced, ragged grid (160 x 12), sigma = 100, 2000 steps;
    float32 u and E: test_fp32_small_signal_groups."""
    skip = FP32_SMALL_SIGNAL["sheet"] if precision == L.FP32 else ()
    assert_parity(_case_errors("sheet", precision), TOL[precision], skip=skip)


@pytest.mark.parametrize("precision", [L.FP64, L.FP32])
def test_kelvin_helmholtz_short_horizon(precision):
    """Config 3 form (shear +-V, density ratio 10, sigma = 1e3, seeded noise) on
    a 136 x 72 grid (interior and edge tiles of the tile kernel) for 40 steps:
    flowing magnetised plasma is linearly unstable in the scheme (growth of
    rho_c through the convection current), so parity is checked over a short
    horizon; float32 E: test_fp32_small_signal_groups."""
    skip = FP32_SMALL_SIGNAL["kh"] if precision == L.FP32 else ()
    assert_parity(_case_errors("kh", precision), TOL[precision], skip=skip)


@pytest.mark.xfail(strict=True, reason="float32 floor of small-signal fields (module docstring): sheet u 5.7e-5, "
                                       "E 1.5e-5 at 2000 steps; KH E 3.7e-5 at 40 steps; 3-D rho_c 2.4e-5 at 10 steps")
@pytest.mark.parametrize("case", ["sheet", "kh", "3d"])
def test_fp32_small_signal_groups(case):
    errs = _case_errors(case, L.FP32)
    print(case, {k: errs[k] for k in FP32_SMALL_SIGNAL[case]})
    assert all(errs[k] <= 1e-5 for k in FP32_SMALL_SIGNAL[case]), errs


@pytest.mark.parametrize("precision", [L.FP64, L.FP32])
def test_three_dimensional_periodic(precision):
    """A 3-D periodic state with every population moving (24 x 20 x 18), the
    3-D periodic step kernel in float64 and float32; short horizon (3-D flows
    with fields are unstable in the scheme within ~15 steps); float32 rho_c:
    test_fp32_small_signal_groups."""
    errs = _case_errors("3d", precision)
    print("3-D periodic", precision, errs)
    assert_parity(errs, TOL[precision], skip=FP32_SMALL_SIGNAL["3d"] if precision == L.FP32 else ())


def test_open_boundaries_fp64():
    """Open y faces with the normal-B fix (the paper's KH boundaries)."""
    F = W.kelvin_helmholtz(48, 40, 1, V=0.1, ratio=3.0, B0=0.1, a=2.0, noise=1e-2, seed=5)
    rng = np.random.default_rng(71)
    F.B[1] += 0.005 * rng.uniform(-1, 1, F.N)
    errs, _ = run_pair(F, 30, L.FP64, bc=(L.PERIODIC, L.PERIODIC, L.OPEN, L.OPEN, L.PERIODIC, L.PERIODIC),
                       sigma=100.0)
    assert_parity(errs, 1e-10)


def test_flux_rope_open_and_driven_fp64():
    """Config 5 form on a small grid: open faces, driven photosphere."""
    F = W.flux_rope(20, 16, 24)
    nl = W.drive_layers_for(24)
    errs, _ = run_pair(F, 25, L.FP64, bc=(L.OPEN, L.OPEN, L.OPEN, L.OPEN, L.DRIVEN, L.OPEN), sigma=500.0,
                       drive_u0=0.05, drive_layers=nl)
    assert_parity(errs, 1e-10)


# float16-deviation storage (f, g as float16 relative deviations, float32
# arithmetic): its bar follows from the float16 resolution, 2^-11 = 4.9e-4 of
# each stored deviation. The large fields (n, p, eps, B) carry it at ~1e-5 of
# their size; u and E are the small signals of the populations (the flow is
# ~1e-3 of a deviation's scale on the current sheet), resolved to ~1e-2. Not
# error-matched with float32 (module docstring: 1e-5): the benchmark reports
# both side by side.
FP16_BAR = {"n": 1e-4, "p": 1e-4, "eps": 1e-4, "B": 1e-4, "u": 3e-2, "E": 3e-2}


def test_fp16_deviation_storage_bar():
    """The reduced current sheet (160 x 12, sigma = 100) over 400 steps within
    the float16-deviation bar."""
    F = W.current_sheet(160, 12, 1, delta=8.0)
    errs, _ = run_pair(F, 400, L.FP16_DEV, sigma=100.0)
    print("fp16 sheet 400 steps", errs)
    assert_parity(errs, 0.0, loose=FP16_BAR)


@pytest.mark.parametrize("precision", [L.FP64, L.FP32])
def test_em_streaming_permutation_bit_exact(precision):
    """With the EM collision switched off, h after n steps is the initial h
    rolled by n lattice hops, bit for bit (ragged 3-D grid)."""
    nx, ny, nz = 37, 11, 6
    N = nx * ny * nz
    rng = np.random.default_rng(72)
    s = L.Solver(L.make_params(nx, ny, nz, sigma=10.0, precision=precision, flags=L.FLAG_NO_EM_COLLISION))
    s.init_fields(0, np.ones(N), np.ones(N), rng.uniform(-0.1, 0.1, (3, N)), rng.uniform(-0.1, 0.1, (3, N)))
    _, _, h0 = s.populations()
    n = 5
    s.step(n)
    _, _, h1 = s.populations()
    hop = L.lattice_tables()["hop"].astype(int)
    for k in range(24):
        expect = np.roll(h0[k].reshape(nz, ny, nx), (n * hop[k][2], n * hop[k][1], n * hop[k][0]), axis=(0, 1, 2))
        assert np.array_equal(h1[k].reshape(nz, ny, nx), expect), k
    assert np.array_equal(h1[24], h0[24])


def test_mass_and_charge_conserved_fp64():
    F = W.kelvin_helmholtz(64, 48, 1, V=0.1, ratio=3.0, B0=0.1, a=2.0, noise=1e-2, seed=9)
    s = L.Solver(L.make_params(F.nx, F.ny, F.nz, sigma=100.0, precision=L.FP64))
    s.init_fields(0, F.n, F.p, F.u, F.B)
    d0 = s.diagnostics()
    s.step(40)
    d1 = s.diagnostics()
    assert abs(d1[0] - d0[0]) < 1e-12 * d0[0]
    assert abs(d1[5] - d0[5]) < 1e-12
    assert d1[8] == 0 and d1[9] == F.N


def test_diagnostics_match_oracle_totals():
    """Sums of N^0 and rho_c of the post-collision state equal the oracle's
    (the g collision conserves N^0 and the h_0 update conserves charge)."""
    F = W.kelvin_helmholtz(40, 32, 1, V=0.3, ratio=3.0, B0=0.1, a=2.0, noise=1e-2, seed=11)
    ref = O.Sim(O.make_params(F.nx, F.ny, 1, sigma=100.0, threads=8))
    ref.init(F.n, F.p, F.u, F.B)
    ref.step(20)
    f, g, h, _ = ref.state()
    lat = O.lattice(ref.P)
    s = L.Solver(L.make_params(F.nx, F.ny, 1, sigma=100.0, precision=L.FP64))
    s.init_fields(0, F.n, F.p, F.u, F.B)
    s.step(20)
    d = s.diagnostics()
    assert abs(d[0] - (lat["p"][:, 0:1] * g).sum()) < 1e-11 * d[0]
    assert abs(d[5] - h.sum()) < 1e-11


@pytest.mark.parametrize("precision", [L.FP32, L.FP16_DEV, L.FP64])
def test_checkpoint_resume_bit_exact(precision):
    """Checkpoint / restore of the raw state (the population groups and pairs
    and the primitive vectors of every storage format) continues bit for bit;
    a blob whose layout tag differs is refused."""
    F = W.kelvin_helmholtz(48, 40, 1, V=0.3, ratio=3.0, B0=0.1, a=2.0, noise=1e-2, seed=13)
    P = L.make_params(F.nx, F.ny, 1, sigma=100.0, precision=precision)
    a = L.Solver(P)
    a.init_fields(0, F.n, F.p, F.u, F.B)
    a.step(20)
    b = L.Solver(P)
    b.init_fields(0, F.n, F.p, F.u, F.B)
    b.step(9)
    blob = b.get_state()
    c = L.Solver(P)
    bad = bytearray(blob)
    bad[1] ^= 0x01  # the layout tag in front of the state
    with pytest.raises(L.LbrmhdError) as e:
        c.set_state(bytes(bad))
    assert e.value.code == L.ERR_BAD_ARG
    c.set_state(blob)
    c.step(11)
    assert np.array_equal(a.moments(), c.moments())
    fa, ga, ha = a.populations()
    fc, gc, hc = c.populations()
    assert np.array_equal(fa, fc) and np.array_equal(ga, gc) and np.array_equal(ha, hc)
    assert c.stats()["steps"] == 20


def test_uniform_state_stays_uniform_fp32():
    N = 40 * 30
    u = np.tile(np.array([[0.2], [-0.1], [0.0]]), N)
    B = np.tile(np.array([[0.1], [0.05], [0.0]]), N)
    s = L.Solver(L.make_params(40, 30, 1, sigma=50.0, precision=L.FP32))
    s.init_fields(0, np.full(N, 1.3), np.full(N, 0.7), u, B)
    m0 = s.moments()
    s.step(50)
    m = s.moments()
    assert np.abs(m - m0).max() < 1e-6
    assert np.all(m.std(axis=1) <= 1e-7 * (1 + np.abs(m).max(axis=1)))


def test_full_size_sampled_step_fp32():
    """Config 2 at its full size (1024 x 1024, sigma = 100, float32) in the
    launch configuration the benchmark times: one GPU step checked at 400
    sampled cells against the oracle's step of the same (GPU) state."""
    nx = ny = 1024
    F = W.current_sheet(nx, ny, 1, delta=8.0)
    s = L.Solver(L.make_params(nx, ny, 1, sigma=100.0, precision=L.FP32))
    s.init_fields(0, F.n, F.p, F.u, F.B)
    s.step(3)
    fc, gc, hc = s.populations()
    m = s.moments()
    prim = np.zeros((O.NPRIM, F.N))
    prim[O.N_] = m[0]
    prim[O.EPS_] = m[2]
    prim[O.U_:O.U_ + 3] = m[3:6]
    prim[O.E_:O.E_ + 3] = m[6:9]
    prim[O.B_:O.B_ + 3] = m[9:12]
    prim[O.RHOC_] = m[12]
    prim[O.J_:O.J_ + 3] = m[13:16]
    rng = np.random.default_rng(73)
    cells = np.unique(np.concatenate([rng.integers(0, F.N, 392), [0, nx - 1, F.N - 1, F.N - nx, 1023 * nx + 5]]))
    ref = O.Sim(O.make_params(nx, ny, 1, sigma=100.0, threads=8))
    _, _, _, pr = ref.update_cells_from(fc, gc, hc, prim, cells)
    s.step(1)
    m1 = s.moments()[:, cells]
    for name, rows in (("n", [0]), ("eps", [2]), ("u", [3, 4, 5]), ("E", [6, 7, 8]), ("B", [9, 10, 11])):
        orows = {"n": [O.N_], "eps": [O.EPS_], "u": [2, 3, 4], "E": [5, 6, 7], "B": [8, 9, 10]}[name]
        a, b = m1[rows], pr[:, orows].T
        nb = np.linalg.norm(b)
        err = np.linalg.norm(a - b) / nb if nb > 0 else np.linalg.norm(a - b)
        assert err <= 1e-5 or np.linalg.norm(a - b) < 1e-9, (name, err)


@functools.lru_cache(maxsize=1)
def _sheet_1024_oracle_moments(steps):
    F = W.current_sheet(1024, 1024, 1, delta=8.0)
    ref = O.Sim(O.make_params(1024, 1024, 1, sigma=100.0, threads=16))
    ref.init(F.n, F.p, F.u, F.B)
    ref.step(steps)
    return ref.moments()


@pytest.mark.parametrize("precision", [L.FP64, L.FP32, L.FP16_DEV])
def test_full_size_multi_step_in_the_benchmark_launch_configuration(precision):
    """Config 2 at its full size (1024 x 1024) in the launch configuration the
    benchmark times: the three runs (sigma = 10, 100, 1000) in one handle, one
    launch per run per step on three streams, replayed from 10-step CUDA
    graphs; 20 steps, the sigma = 100 run against the oracle over every cell:
    float64 and float32 every group within their bars, float16-deviation
    storage within FP16_BAR."""
    torch = pytest.importorskip("torch")
    nx = ny = 1024
    F = W.current_sheet(nx, ny, 1, delta=8.0)
    s = L.Solver([L.make_params(nx, ny, 1, sigma=sg, precision=precision) for sg in (10.0, 100.0, 1000.0)],
                 stream=torch.cuda.current_stream())
    for r in range(3):
        s.init_fields(r, F.n, F.p, F.u, F.B)
    s.set_schedule(kind=L.SCHED_PER_RUN, streams=3, graph_steps=10)
    s.step(20)
    mg = s.moments(1)
    st = s.status()
    s.close()
    assert st["rc"] == L.OK, st
    errs = rel_errors(mg, _sheet_1024_oracle_moments(20))
    print("full size 20 steps", {L.FP64: "FP64", L.FP32: "FP32", L.FP16_DEV: "FP16_DEV"}[precision], errs)
    if precision == L.FP16_DEV:
        assert_parity(errs, 0.0, loose=FP16_BAR)
    else:
        assert_parity(errs, TOL[precision])
