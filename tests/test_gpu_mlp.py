"""The learned recovery seed on the GPU, through the C ABI, against the float64
reference of oracle/mlp_ref.py and the FP64 oracle of the method.

- training samples written by the step kernel = features of the oracle's
  streamed moments and the oracle's recovered primitives (float64 run);
- float32 gradient and Adam training = float64 back-propagation and Adam on
  the same mini-batch rows;
- tensor-core inference = the bf16-rounded float64 forward pass;
- a run seeded by a network trained on the GPU from the method's own samples
  matches the oracle like the plain run does (the seed only starts the
  eigen-solve), and needs fewer iterations than the same solve without history.
"""
import numpy as np
import pytest

import oracle as O
from oracle import mlp_ref as M
from paper_1508_03452_gb300 import lbrmhd as L
from paper_1508_03452_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _torch():
    return pytest.importorskip("torch")


def _solver(F, precision, recovery, flags=0, **kw):
    torch = _torch()
    s = L.Solver(L.make_params(F.nx, F.ny, F.nz, precision=precision, recovery=recovery, flags=flags, **kw),
                 stream=torch.cuda.current_stream())
    s.init_fields(0, F.n, F.p, F.u, F.B, F.E)
    return s


def _training_fields():
    return [(W.kelvin_helmholtz(128, 96, 1, V=0.2, ratio=10.0, B0=0.1, a=2.0, noise=1e-3, seed=s), 1e3)
            for s in (11, 12)] + [(W.current_sheet(256, 32, 1, delta=8.0), 100.0)]


def _collect(cases, steps=40, every=4, precision=L.FP32):
    """Samples the method writes while it runs (cold-seeded recovery)."""
    torch = _torch()
    out = []
    for F, sigma in cases:
        s = _solver(F, precision, L.RECOVERY_COLD, sigma=sigma)
        buf = torch.full((F.N, L.MLP_ROW), float("nan"), dtype=torch.float32, device="cuda")
        s.set_mlp_samples(0, buf)
        for t in range(steps):
            s.step(1)
            if t % every == every - 1:
                out.append(buf.clone())
        s.close()
    data = torch.cat(out)
    return data[torch.isfinite(data).all(1)].contiguous()


@pytest.fixture(scope="module")
def trained():
    """A network trained on the GPU from the method's own samples (float32
    runs of the current-sheet and Kelvin-Helmholtz set-ups)."""
    torch = _torch()
    data = _collect(_training_fields())
    P = torch.tensor(W.mlp_init_params(1), device="cuda")
    adam = torch.zeros(2 * L.MLP_NPARAM, device="cuda")
    losses = L.mlp_train(P, adam, data, 3000, 1024, 1e-3, seed=7).cpu().numpy()
    return P, data, losses


def test_samples_match_oracle_streamed_moments():
    """Features and targets the float64 step kernel writes = features of the
    oracle's streamed moments (Eqs. Cal_T, Cal_N) and its recovered beta, eps."""
    torch = _torch()
    F = W.kelvin_helmholtz(24, 20, 1, V=0.2, ratio=10.0, B0=0.1, a=2.0, noise=1e-3, seed=5)
    kw = dict(sigma=1e3, alpha=0.0)
    Po = O.make_params(F.nx, F.ny, F.nz, **kw)
    ref = O.Sim(O.make_params(F.nx, F.ny, F.nz, threads=1, **kw))
    ref.init(F.n, F.p, F.u, F.B, F.E)
    m0 = ref.moments()
    fc, gc, hc = ref.post_collision()
    fs = np.stack([O.stream_population(Po, i, fc[i]) for i in range(19)])
    gs = np.stack([O.stream_population(Po, i, gc[i]) for i in range(19)])
    ref.step(1)
    m1 = ref.moments()
    want = np.zeros((F.N, M.ROW))
    for c in range(F.N):
        T, N, _, _, _ = O.moments(Po, fs[:, c], gs[:, c], hc[:, c])
        want[c, :M.N_IN] = M.features(T, N, m0[6:9, c], m0[9:12, c])
        want[c, M.N_IN:] = M.targets(m1[3:6, c], m1[2, c], 1.0, T[0, 0])

    s = _solver(F, L.FP64, L.RECOVERY_COLD, **kw)
    buf = torch.full((F.N, L.MLP_ROW), float("nan"), dtype=torch.float32, device="cuda")
    s.set_mlp_samples(0, buf)
    s.step(1)
    got = buf.cpu().numpy().astype(np.float64)
    s.close()
    # relative to each column's scale; columns that are physically zero in
    # this in-plane problem (T^0z, beta_z) hold round-off on both sides and
    # are held to an absolute floor instead
    scale = np.maximum(np.abs(want).max(0), 1e-9)
    err = np.abs(got - want).max(0) / scale
    assert np.all(np.isfinite(got))
    assert err.max() < 2e-6, err  # float32 storage of float64 values


def test_plain_run_with_sample_buffer_writes_samples():
    torch = _torch()
    F = W.current_sheet(64, 8, 1, delta=4.0)
    s = _solver(F, L.FP32, L.RECOVERY_PLAIN, sigma=100.0)
    buf = torch.full((F.N, L.MLP_ROW), float("nan"), dtype=torch.float32, device="cuda")
    s.set_mlp_samples(0, buf)
    s.step(2)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(buf).all())
    assert float(buf[:, 19].min()) == 1.0 == float(buf[:, 19].max())
    s.set_mlp_samples(0, None)
    buf.fill_(float("nan"))
    s.step(1)
    torch.cuda.synchronize()
    assert bool(torch.isnan(buf).all())
    s.close()


def test_learned_seed_requires_weights():
    F = W.current_sheet(32, 8, 1, delta=4.0)
    s = _solver(F, L.FP32, L.RECOVERY_MLP, sigma=100.0)
    with pytest.raises(L.LbrmhdError) as e:
        s.step(1)
    assert e.value.code == L.ERR_STATE
    s.close()


def test_gradient_matches_float64_backprop():
    torch = _torch()
    r = np.random.default_rng(3)
    n = 3000
    X = r.normal(0, 0.5, size=(n, M.N_IN))
    X[:, 19] = 1
    Y = r.normal(0, 0.2, size=(n, M.N_OUT))
    data = np.concatenate([X, Y], 1).astype(np.float32)
    P = W.mlp_init_params(2)
    loss, g = L.mlp_grad(torch.tensor(P, device="cuda"), torch.tensor(data, device="cuda"))
    Lw, gw = M.loss_and_grad(P.astype(np.float64), data[:, :20].astype(np.float64), data[:, 20:].astype(np.float64))
    g = g.cpu().numpy().astype(np.float64)
    assert loss == pytest.approx(Lw, rel=1e-5)
    o = 0
    for name, shape in M.SHAPES:
        k = int(np.prod(shape))
        e = np.linalg.norm(g[o:o + k] - gw[o:o + k]) / np.linalg.norm(gw[o:o + k])
        assert e < 1e-5, (name, e)
        o += k


def test_training_matches_float64_adam_and_is_reproducible():
    torch = _torch()
    r = np.random.default_rng(4)
    n = 2000
    X = r.uniform(-1, 1, size=(n, M.N_IN))
    X[:, 19] = 1
    Y = np.stack([np.sin(X[:, 0]), X[:, 1] * X[:, 2], 0.1 * X[:, 3], np.cos(X[:, 4]) - 1], 1)
    data = np.concatenate([X, Y], 1).astype(np.float32)
    P0 = W.mlp_init_params(5)
    steps, batch, lr, seed = 6, 256, 1e-3, 99
    runs = []
    for _ in range(2):
        P = torch.tensor(P0, device="cuda")
        adam = torch.zeros(2 * L.MLP_NPARAM, device="cuda")
        losses = L.mlp_train(P, adam, torch.tensor(data, device="cuda"), steps, batch, lr, seed=seed)
        runs.append((P.cpu().numpy(), losses.cpu().numpy()))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    Pw, _, _, lw = M.train(P0.astype(np.float64), np.zeros(M.NPARAM), np.zeros(M.NPARAM),
                           data.astype(np.float64), steps, batch, lr, seed)
    assert np.allclose(runs[0][1], lw, rtol=1e-5, atol=0)
    step_gpu, step_ref = runs[0][0] - P0, Pw - P0
    assert np.linalg.norm(step_gpu - step_ref) < 1e-3 * np.linalg.norm(step_ref)


def test_inference_matches_bf16_forward(trained):
    torch = _torch()
    P, data, _ = trained
    feats = data[:: max(1, data.shape[0] // 20000), :L.MLP_NFEAT].contiguous()
    blob = L.mlp_pack(P)
    y = L.mlp_infer(blob, feats).cpu().numpy()
    want = M.forward_bf16(P.cpu().numpy().astype(np.float64), feats.cpu().numpy().astype(np.float64))
    d = np.abs(y - want).max(1)
    scale = np.abs(want).max()
    # float32 accumulation order may flip a bf16 rounding of a hidden unit
    assert np.quantile(d, 0.99) <= 1e-5 * scale and d.max() <= 1e-2 * scale, (np.quantile(d, 0.99), d.max(), scale)
    # and the bf16 path stays close to the float64 network
    full = M.forward(P.cpu().numpy().astype(np.float64), feats.cpu().numpy().astype(np.float64))
    assert np.abs(y - full).max() <= 0.05 * scale


def test_trained_network_fits_the_recovery(trained):
    P, data, losses = trained
    assert losses[-100:].mean() < 0.02 * losses[:10].mean(), (losses[:10].mean(), losses[-100:].mean())
    torch = _torch()
    y = L.mlp_infer(L.mlp_pack(P), data[:, :L.MLP_NFEAT].contiguous())
    err = (y[:, :3] - data[:, 20:23]).norm(dim=1)
    beta = data[:, 20:23].norm(dim=1)
    assert float(err.mean()) < 0.1 * float(beta.mean()), (float(err.mean()), float(beta.mean()))


@pytest.mark.parametrize("precision", [L.FP64, L.FP32])
def test_learned_seed_run_parity(trained, precision):
    """A held-out Kelvin-Helmholtz run seeded by the network matches the oracle
    with the plain run's bars (the converged solve is the method's)."""
    from test_gpu_parity import FP32_SMALL_SIGNAL, TOL, assert_parity, rel_errors
    P, _, _ = trained
    F = W.kelvin_helmholtz(136, 72, 1, V=0.2, ratio=10.0, B0=0.1, a=2.0, noise=1e-3, seed=3)
    ref = O.Sim(O.make_params(F.nx, F.ny, F.nz, sigma=1e3, threads=8))
    ref.init(F.n, F.p, F.u, F.B, F.E)
    ref.step(40)
    s = _solver(F, precision, L.RECOVERY_MLP, sigma=1e3)
    s.set_mlp_weights(P)
    s.step(40)
    errs = rel_errors(s.moments(), ref.moments())
    st = s.stats()
    s.close()
    assert st["recover_fail"] == 0, st
    print("learned seed KH", errs)
    assert_parity(errs, TOL[precision], skip=FP32_SMALL_SIGNAL["kh"] if precision == L.FP32 else ())


def _iterations(F, sigma, recovery, flags, P=None, steps=20, precision=L.FP32):
    s = _solver(F, precision, recovery, flags, sigma=sigma)
    if P is not None:
        s.set_mlp_weights(P)
    s.step(steps)
    st = s.stats()
    m = s.moments()
    s.close()
    assert st["recover_fail"] == 0, st
    return st["iter_total"] / (steps * F.N), m


@pytest.mark.parametrize("flags", [L.FLAG_UNSHIFTED_POWER, 0])
def test_learned_seed_gain(trained, flags):
    """What the trained network gains: mean eigen-solve iterations per cell and
    step on a held-out run at the same tolerance, against zero velocity (the
    solve without history) and against the library's default, the previous
    step's velocity (RECOVERY_PLAIN, the method without the network). The
    network beats the cold start; it does not beat the previous-step seed,
    which in a time-stepping run is already within one step of the answer
    (measured: plain power method 10.2 vs 7.7 iterations, shifted 3.73 vs
    3.63), and the test records that. The converged fields agree to the
    solve's tolerance."""
    P, _, _ = trained
    F = W.kelvin_helmholtz(128, 96, 1, V=0.2, ratio=10.0, B0=0.1, a=2.0, noise=1e-3, seed=31)
    it_cold, m_cold = _iterations(F, 1e3, L.RECOVERY_COLD, flags)
    it_mlp, m_mlp = _iterations(F, 1e3, L.RECOVERY_MLP, flags, P)
    it_prev, _ = _iterations(F, 1e3, L.RECOVERY_PLAIN, flags)
    msg = (f"flags={flags}: iterations/cell cold {it_cold:.3f} learned {it_mlp:.3f} "
           f"previous-step (RECOVERY_PLAIN) {it_prev:.3f}")
    print(msg)
    assert it_mlp < (0.9 if flags else 1.0) * it_cold, msg
    # no gain over the method without the network (within 10 %)
    assert it_mlp >= 0.9 * it_prev, msg
    rows = [3, 4, 5]
    d = np.linalg.norm(m_mlp[rows] - m_cold[rows]) / np.linalg.norm(m_cold[rows])
    assert d < 1e-4, d


def test_recovery_failures_do_not_depend_on_the_seed(trained):
    """Why the learned seed has no retry job: on a Kelvin-Helmholtz run that
    breaks down (V = 0.5 c, density ratio 10, the paper's readings), the first
    failing step and the cells failing there are the same whether the
    eigen-solve starts from the previous step's velocity, from rest or from
    the trained network (measured: step 16, 166 cells, for all three). The
    streamed moments there have no physical solution, whatever the start."""
    P, _, _ = trained
    F = W.kelvin_helmholtz(256, 256, 1, V=0.5, ratio=10.0, B0=0.1, a=2.0, noise=1e-3, seed=3)
    first = {}
    for name, rec in (("prev", L.RECOVERY_PLAIN), ("cold", L.RECOVERY_COLD), ("learned", L.RECOVERY_MLP)):
        s = _solver(F, L.FP32, rec, sigma=1e3)
        if rec == L.RECOVERY_MLP:
            s.set_mlp_weights(P)
        for t in range(1, 41):
            s.step(1)
            f = s.stats()["recover_fail"]
            if f:
                first[name] = (t, f)
                break
        s.close()
    print("first failing step and failed cells:", first)
    assert set(first) == {"prev", "cold", "learned"}, first
    # the three kernels are compiled separately (float rounding may differ in
    # the last bit before the breakdown): same step, counts within 10 %
    assert first["prev"][0] == first["cold"][0] == first["learned"][0], first
    counts = [v[1] for v in first.values()]
    assert max(counts) <= 1.1 * min(counts), first


@pytest.mark.parametrize("recovery", [L.RECOVERY_PLAIN, L.RECOVERY_COLD])
def test_iteration_histogram_matches_counters(recovery):
    """The histogram counts every converged cell update once and, below its
    overflow bin, reproduces the iteration sum and maximum."""
    F = W.kelvin_helmholtz(96, 40, 1, V=0.2, ratio=10.0, B0=0.1, a=2.0, noise=1e-3, seed=8)
    steps = 7
    s = _solver(F, L.FP32, recovery, flags=L.FLAG_UNSHIFTED_POWER, sigma=1e3)
    s.step(steps)
    hist, st = s.iteration_histogram(0), s.stats(0)
    s.close()
    assert hist.sum() + st["recover_fail"] == steps * F.N
    k = np.arange(1, L.NHIST + 1)
    if hist[-1] == 0:
        assert int((k * hist).sum()) == st["iter_total"]
        assert int(k[hist > 0].max()) == st["iter_max"]
    else:
        assert int((k[:-1] * hist[:-1]).sum()) + L.NHIST * int(hist[-1]) <= st["iter_total"]
