"""CPU checks of the C-ABI library: it builds, loads and exports every symbol
its header declares; its compiled-in lattice tables agree with the oracle's
independently written ones; and without a GPU it refuses to run (no CPU
fallback)."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1508_03452_gb300 import lbrmhd as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lbrmhd_\w+)\s*\(", text))
    return sorted(names)


def test_header_symbols_are_exported():
    lib = L.load()
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(L.EXPORTED) == set(names)


def test_learned_seed_layout_constants_need_no_gpu():
    from oracle import mlp_ref as M
    lib = L.load()
    assert lib.lbrmhd_mlp_nparams() == L.MLP_NPARAM == M.NPARAM
    # bf16 weights in fragment order (W1 64 x 32 with zero-padded inputs, W2 and
    # W3 64 x 64, W4 8 x 64 with zero-padded outputs), then 200 float32 biases
    assert lib.lbrmhd_mlp_blob_bytes() == 2 * (64 * 32 + 2 * 64 * 64 + 8 * 64) + 4 * 200
    assert lib.lbrmhd_mlp_pack(None, None, None) == L.ERR_BAD_ARG
    assert lib.lbrmhd_mlp_infer(None, None, 1, None, None) == L.ERR_BAD_ARG
    assert lib.lbrmhd_mlp_grad(None, None, 1, None, None) == L.ERR_BAD_ARG
    assert lib.lbrmhd_set_mlp_weights(None, None) == L.ERR_BAD_ARG
    assert lib.lbrmhd_set_mlp_samples(None, 0, None) == L.ERR_BAD_ARG
    assert lib.lbrmhd_get_iteration_histogram(None, 0, None) == L.ERR_BAD_ARG
    assert lib.lbrmhd_set_schedule(None, None) == L.ERR_BAD_ARG
    assert lib.lbrmhd_get_schedule(None, None) == L.ERR_BAD_ARG
    assert lib.lbrmhd_autotune(None, 1, None, None) == L.ERR_BAD_ARG
    assert lib.lbrmhd_reconnection_rate(None, 0, 0, 1, 1.0, None) == L.ERR_BAD_ARG


def test_lattice_tables_match_oracle():
    t = L.lattice_tables()
    lat = O.lattice(O.make_params(c=1.0))
    assert np.array_equal(t["chat"], lat["chat"])
    assert np.allclose(t["w"], lat["w"], rtol=0, atol=1e-15)
    assert np.allclose(t["wg"], lat["wg"], rtol=0, atol=1e-15)
    assert np.array_equal(t["hop"], lat["hop"])
    assert np.allclose(t["e_over_c"], lat["e"], rtol=0, atol=1e-15)
    assert np.allclose(t["b"], lat["b"], rtol=0, atol=1e-15)


def test_bad_parameters_are_rejected():
    with pytest.raises(L.LbrmhdError) as e:
        L.Solver(L.make_params(0, 4, 1))
    assert e.value.code == L.ERR_BAD_ARG
    with pytest.raises(L.LbrmhdError) as e:
        L.Solver(L.make_params(8, 4, 4, bc=(L.DRIVEN, L.DRIVEN, 0, 0, 0, 0)))
    assert e.value.code == L.ERR_BAD_ARG
    with pytest.raises(L.LbrmhdError) as e:
        L.Solver(L.make_params(8, 4, 4, bc=(L.OPEN, L.PERIODIC, 0, 0, 0, 0)))
    assert e.value.code == L.ERR_BAD_ARG
    # above 2^29 cells the step kernel's 32-bit stencil offsets (x4 per group vector) would overflow
    with pytest.raises(L.LbrmhdError) as e:
        L.Solver(L.make_params(32768, 16385, 1))
    assert e.value.code == L.ERR_BAD_ARG
    assert "2^29" in str(e.value)
    # the photospheric body force: needs forced layers, replaces the DRIVEN
    # face, finite values; unknown flags are refused
    for kw in (dict(drive_f0=0.05, drive_layers=0), dict(drive_f0=0.05, drive_layers=2,
                                                       bc=(L.OPEN,) * 4 + (L.DRIVEN, L.OPEN)),
               dict(drive_f0=float("nan"), drive_layers=2), dict(drive_vmax=float("inf")), dict(flags=64)):
        with pytest.raises(L.LbrmhdError) as e:
            L.Solver(L.make_params(8, 8, 8, **kw))
        assert e.value.code == L.ERR_BAD_ARG, kw


def test_valid_options_pass_validation():
    """Valid force and Gauss-charge parameters pass the parameter check: with
    no GPU the creation then fails on the device, not on the arguments."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    for kw in (dict(drive_f0=0.05, drive_layers=2, drive_vmax=0.75, bc=(L.OPEN,) * 6),
               dict(flags=L.FLAG_GAUSS_CHARGE | L.FLAG_ONE_PASS_RECOVERY)):
        with pytest.raises(L.LbrmhdError) as e:
            L.Solver(L.make_params(8, 8, 8, **kw))
        assert e.value.code == L.ERR_CUDA, kw
    with pytest.raises(L.LbrmhdError) as e:  # the largest grid (2^29 cells)
        L.Solver(L.make_params(32768, 16384, 1))
    assert e.value.code == L.ERR_CUDA
    lib = L.load()
    assert lib.lbrmhd_init_fields_relaxed(None, 0, None, None, None, None, 10, 1e-6, None, None) == L.ERR_BAD_ARG


def test_no_cpu_fallback_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(L.LbrmhdError) as e:
        L.Solver(L.make_params(8, 8, 1))
    assert e.value.code == L.ERR_CUDA
