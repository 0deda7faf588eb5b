"""Batched launches, CUDA-graph replay and the autotuner, through the C ABI.

The schedule only regroups the same cell updates into launches. In float64
every schedule gives bit-identical states; in float32 the per-run and batched
kernels are compiled separately (floating-point contraction may differ in the
last bit), and the self-consistent recovery's stopping test can turn that bit
into one more or one fewer field iteration, so float32 schedules agree to the
recovery tolerance. The autotuner's dry steps must leave the state and the
counters untouched; and a batch of uneven runs must match the FP64 oracle run
by run.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_1508_03452_gb300 import lbrmhd as L
from paper_1508_03452_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _torch():
    return pytest.importorskip("torch")


def uneven_batch():
    """Runs of uneven (and ragged) grids, 2-D and 3-D, periodic and open, with
    plain and cold-seeded recovery: every kernel group of the batch path."""
    specs = []
    for i, (nx, ny, V, ratio, sigma) in enumerate([(40, 24, 0.1, 1.0, 100.0), (64, 48, 0.2, 3.0, 1e3),
                                                   (96, 8, 0.1, 10.0, 30.0), (130, 20, 0.15, 3.0, 1e4)]):
        F = W.kelvin_helmholtz(nx, ny, 1, V=V, ratio=ratio, B0=0.1, a=2.0, noise=1e-3, seed=40 + i)
        specs.append((F, dict(sigma=sigma)))
    F = W.current_sheet(48, 32, 1, delta=4.0)
    specs.append((F, dict(sigma=100.0, bc=(L.OPEN, L.OPEN, L.PERIODIC, L.PERIODIC, L.PERIODIC, L.PERIODIC))))
    rng = np.random.default_rng(9)
    nx, ny, nz = 16, 12, 10
    N = nx * ny * nz
    u = np.zeros((3, N))
    u[0] = 0.02 * rng.uniform(-1, 1, N)
    B = np.zeros((3, N))
    B[2] = 0.05
    specs.append((W.Fields(nx, ny, nz, 1.0 + 0.02 * rng.uniform(size=N), np.ones(N), u, B), dict(sigma=50.0)))
    F = W.kelvin_helmholtz(56, 16, 1, V=0.1, ratio=3.0, B0=0.1, a=2.0, noise=1e-3, seed=77)
    specs.append((F, dict(sigma=1e3, recovery=L.RECOVERY_COLD)))
    return specs


def make_solver(specs, precision):
    torch = _torch()
    params = [L.make_params(F.nx, F.ny, F.nz, precision=precision, **kw) for F, kw in specs]
    s = L.Solver(params, stream=torch.cuda.current_stream())
    for r, (F, _) in enumerate(specs):
        s.init_fields(r, F.n, F.p, F.u, F.B, F.E)
    return s


def snapshot(s, nruns):
    return [np.concatenate([np.concatenate(s.populations(r)).ravel(), s.moments(r).ravel()]) for r in range(nruns)]


SCHEDULES = [dict(kind=L.SCHED_PER_RUN), dict(kind=L.SCHED_PER_RUN, streams=3)] + [
    dict(kind=L.SCHED_BATCH, bx=bx, waves=w, order=o) for bx, w, o in itertools.product((128, 64, 32), (0, 1), (0, 1))]


@pytest.mark.parametrize("precision", [L.FP64, L.FP32])
def test_every_schedule_is_bit_identical(precision):
    specs = uneven_batch()
    steps = 9
    ref = None
    for sc in SCHEDULES + [dict(kind=L.SCHED_BATCH, bx=64, waves=1, order=1, graph_steps=4),
                           dict(kind=L.SCHED_PER_RUN, graph_steps=2),
                           dict(kind=L.SCHED_PER_RUN, streams=4, graph_steps=4)]:
        s = make_solver(specs, precision)
        s.set_schedule(**sc)
        s.step(steps)  # odd: graphs of 4 or 2 steps, then direct steps
        snap = snapshot(s, len(specs))
        st = [s.stats(r) for r in range(len(specs))]
        s.close()
        if ref is None:
            ref = (snap, st)
            continue
        for r in range(len(specs)):
            if precision == L.FP64:
                assert np.array_equal(snap[r], ref[0][r]), (sc, r)
                assert st[r] == ref[1][r], (sc, r)
            else:
                _assert_close(snap[r], ref[0][r], (sc, r))
                assert st[r]["recover_fail"] == ref[1][r]["recover_fail"], (sc, r)


def _assert_close(a, b, what):
    """float32 states equal to the recovery tolerance (1e-5 of the array's scale)."""
    assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max(), what


def test_default_schedule_and_validation():
    specs = uneven_batch()[:2]
    s = make_solver(specs, L.FP32)
    sc = s.schedule()
    assert (sc.kind, sc.streams, sc.graph_steps) == (L.SCHED_PER_RUN, 1, 0)
    for bad in (dict(kind=L.SCHED_BATCH, bx=48), dict(kind=7), dict(kind=L.SCHED_PER_RUN, streams=0),
                dict(kind=L.SCHED_PER_RUN, streams=33), dict(kind=L.SCHED_BATCH, waves=9),
                dict(kind=L.SCHED_BATCH, graph_steps=-1)):
        with pytest.raises(L.LbrmhdError):
            s.set_schedule(**bad)
    assert s.schedule().as_dict() == sc.as_dict()
    s.close()


def test_batch_matches_oracle_run_by_run():
    """A batched FP64 step of uneven runs = the oracle stepping each run alone."""
    from test_gpu_parity import BC_ORC, rel_errors
    specs = uneven_batch()
    steps = 6
    s = make_solver(specs, L.FP64)
    s.set_schedule(kind=L.SCHED_BATCH, bx=64, waves=1, order=1, graph_steps=3)
    s.step(steps)
    for r, (F, kw) in enumerate(specs):
        okw = {k: v for k, v in kw.items() if k == "sigma"}
        bc = kw.get("bc", (L.PERIODIC,) * 6)
        ref = O.Sim(O.make_params(F.nx, F.ny, F.nz, bc=tuple(BC_ORC[b] for b in bc), threads=8, **okw))
        ref.init(F.n, F.p, F.u, F.B, F.E)
        ref.step(steps)
        errs = rel_errors(s.moments(r), ref.moments())
        bad = {k: v for k, v in errs.items() if v is not None and not v <= 1e-10}
        assert not bad, (r, errs)
    s.close()


def test_autotune_leaves_state_untouched_and_picks_a_schedule(tmp_path, monkeypatch):
    specs = uneven_batch()
    n = len(specs)
    a = make_solver(specs, L.FP32)
    a.step(2)
    before = snapshot(a, n)
    st_before = [a.stats(r) for r in range(n)]
    h_before = [a.iteration_histogram(r) for r in range(n)]
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("LBRMHD_TUNE_CACHE", str(cache))
    a.set_schedule(kind=L.SCHED_PER_RUN, graph_steps=3)
    best, ms = a.autotune(trials=2)
    assert ms > 0 and best.graph_steps == 3
    assert a.schedule().as_dict() == best.as_dict()
    assert all(np.array_equal(x, y) for x, y in zip(snapshot(a, n), before))
    assert [a.stats(r) for r in range(n)] == st_before
    assert all(np.array_equal(a.iteration_histogram(r), h) for r, h in enumerate(h_before))
    # continuing after tuning (on the schedule it picked) = a run that was never tuned
    a.step(5)
    b = make_solver(specs, L.FP32)
    b.step(7)
    for x, y in zip(snapshot(a, n), snapshot(b, n)):
        _assert_close(x, y, "after tuning")
    # a second handle of the same batch takes the cached schedule without timing
    lines = cache.read_text().splitlines()
    assert len(lines) == 1
    best2, ms2 = b.autotune(trials=2)
    assert best2.as_dict() | {"graph_steps": 3} == best.as_dict() and ms2 == pytest.approx(ms, rel=1e-5)
    assert len(cache.read_text().splitlines()) == 1
    a.close()
    b.close()


def test_checkpoint_resume_with_graphs_is_bit_exact():
    specs = uneven_batch()
    n = len(specs)
    sched = dict(kind=L.SCHED_BATCH, bx=128, waves=1, order=0, graph_steps=4)
    a = make_solver(specs, L.FP32)
    a.set_schedule(**sched)
    a.step(13)
    blob = a.get_state()
    a.step(11)
    b = make_solver(specs, L.FP32)
    b.set_schedule(**sched)
    b.set_state(blob)
    b.step(11)
    assert all(np.array_equal(x, y) for x, y in zip(snapshot(a, n), snapshot(b, n)))
    assert [a.stats(r) for r in range(n)] == [b.stats(r) for r in range(n)]
    a.close()
    b.close()


def test_learned_seed_runs_batched_match_per_run():
    """The learned-seed kernel variant in a batch (weights set after the runs
    were initialised) = the same runs launched one by one."""
    torch = _torch()
    specs = uneven_batch()[:3]
    specs = [(F, dict(kw, recovery=L.RECOVERY_MLP)) for F, kw in specs[:2]] + [specs[2]]
    P = torch.tensor(W.mlp_init_params(3), device="cuda")
    out = []
    for sc in (dict(kind=L.SCHED_PER_RUN), dict(kind=L.SCHED_BATCH, bx=32, waves=1, order=1, graph_steps=2)):
        s = make_solver(specs, L.FP32)
        s.set_schedule(**sc)
        s.set_mlp_weights(P)
        s.step(5)
        out.append((snapshot(s, len(specs)), [s.stats(r) for r in range(len(specs))]))
        assert all(st["recover_fail"] == 0 for st in out[-1][1])
        s.close()
    for x, y in zip(out[0][0], out[1][0]):
        _assert_close(x, y, "learned seed")


def periodic_batch():
    """Uneven periodic 2-D runs of one kernel variant: what the persistent
    schedule (one cooperative launch for many steps) accepts."""
    specs = []
    for i, (nx, ny, V, ratio, sigma) in enumerate([(40, 24, 0.1, 1.0, 100.0), (64, 48, 0.2, 3.0, 1e3),
                                                   (96, 8, 0.1, 10.0, 30.0), (130, 20, 0.15, 3.0, 1e4),
                                                   (256, 64, 0.1, 3.0, 1e3)]):
        F = W.kelvin_helmholtz(nx, ny, 1, V=V, ratio=ratio, B0=0.1, a=2.0, noise=1e-3, seed=60 + i)
        specs.append((F, dict(sigma=sigma)))
    return specs


@pytest.mark.parametrize("precision", [L.FP64, L.FP32])
def test_persistent_schedule_matches_per_run(precision):
    """K steps in one cooperative launch (grid barrier between steps), directly
    and replayed from graphs, = one launch per run per step."""
    specs = periodic_batch()
    n = len(specs)
    out = []
    for sc in (dict(kind=L.SCHED_PER_RUN), dict(kind=L.SCHED_PERSISTENT, bx=64, order=1),
               dict(kind=L.SCHED_PERSISTENT, bx=128, order=0, graph_steps=4)):
        s = make_solver(specs, precision)
        s.set_schedule(**sc)
        s.step(9)
        out.append((snapshot(s, n), [s.stats(r) for r in range(n)], s.status()))
        s.close()
    for snap, st, status in out[1:]:
        assert status["rc"] == L.OK and status["bits"] == 0, status
        for r in range(n):
            if precision == L.FP64:
                assert np.array_equal(snap[r], out[0][0][r]), r
            else:
                _assert_close(snap[r], out[0][0][r], r)
            assert st[r]["recover_fail"] == out[0][1][r]["recover_fail"] == 0


def test_persistent_schedule_refuses_runs_it_cannot_step():
    """Open faces need a boundary pass between steps, and a 3-D run a different
    kernel variant: the persistent schedule refuses such handles."""
    s = make_solver(uneven_batch(), L.FP32)
    s.set_schedule(kind=L.SCHED_PERSISTENT)
    with pytest.raises(L.LbrmhdError) as e:
        s.step(2)
    assert e.value.code == L.ERR_BAD_ARG
    s.close()


def test_grid_barrier_wait_gives_up():
    """The persistent launch's grid barrier waits with a limit: made to wait for
    an arrival that never comes, every block gives up and raises the status
    bit, the call reports TIMEOUT, and the handle stays usable."""
    import time

    s = make_solver(periodic_batch()[:1], L.FP32)
    lib = L.load()
    assert lib.lbrmhd_barrier_selftest(s._h, 0, 1.0) == L.OK
    t0 = time.perf_counter()
    rc = lib.lbrmhd_barrier_selftest(s._h, 1, 0.05)
    assert rc == L.ERR_TIMEOUT, lib.lbrmhd_last_error(s._h)
    assert time.perf_counter() - t0 < 5.0
    s.step(3)
    assert s.status()["rc"] == L.OK
    s.close()
