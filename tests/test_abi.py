"""CPU checks of the C ABI: the library builds, loads, and exports every entry
point that include/adg.h declares; argument validation needs no GPU."""
import ctypes
import os
import re

import pytest

from paper_1406_7416_gb300 import adg, build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "adg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(adg_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return adg.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(adg.SYMBOLS)


def test_binding_constants_match_the_header():
    """Every #define of include/adg.h that the binding names (ADG_X as adg.X)
    has the header's value."""
    txt = open(os.path.join(ROOT, "include", "adg.h")).read()
    defs = dict(re.findall(r"#define ADG_([A-Z0-9_]+)\s+(-?\d+)\b", txt))
    assert len(defs) > 30
    checked = 0
    for name, val in defs.items():
        if hasattr(adg, name):
            assert getattr(adg, name) == int(val), name
            checked += 1
    assert checked >= 25
    for opt in ("OPT_PREDICTOR", "OPT_SUBCELL_REGISTERS", "PREC_MIXED_TF32"):
        assert opt in defs and hasattr(adg, opt), opt


@pytest.mark.parametrize("dim,N,gamma,bc,prec", [
    (1, 3, 1.4, [0, 0], 0),            # bad dimension
    (2, 0, 1.4, [0, 0, 0, 0], 0),      # N out of range
    (2, 10, 1.4, [0, 0, 0, 0], 0),
    (3, 4, 1.4, [0] * 6, 0),           # 3D limited to N <= 3
    (2, 3, 1.0, [0, 0, 0, 0], 0),      # gamma <= 1
    (2, 3, 1.4, [0, 1, 0, 0], 0),      # unpaired periodic face
    (2, 3, 1.4, [0, 0, 0, 0], 7),      # unknown precision
])
def test_create_rejects_bad_arguments(lib, dim, N, gamma, bc, prec):
    g = adg.AdgGrid()
    g.dim = dim
    for k in range(3):
        g.n[k] = 4
        g.dx[k] = 0.1
    bcs = (ctypes.c_int * 6)(*(bc + [0] * (6 - len(bc))))
    h = ctypes.c_void_p()
    assert lib.adg_create(ctypes.byref(g), N, gamma, bcs, prec, ctypes.byref(h)) == adg.ERR_ARG
    assert not h.value


def test_create_and_destroy_without_device_work(lib):
    s = adg.Solver(2, (5, 3), (0, 0), (0.2, 0.3), (1, 1, 0, 0), 3)
    assert (s.cells, s.nvar, s.nodes, s.subcells) == (15, 4, 16, 49)
    with pytest.raises(adg.AdgError):
        s.step(0.1)            # nothing loaded
    with pytest.raises(adg.AdgError):
        s.set_option(99, 1.0)
    s.close()


@pytest.mark.parametrize("key,bad,good", [
    (adg.OPT_DMP_EPS, -1e-3, 1e-3),
    (adg.OPT_DMP_FLOOR, float("nan"), 1e-4),
    (adg.OPT_PICARD_ITERS, 0, 6),
    (adg.OPT_PICARD_ITERS, 65, 64),
    (adg.OPT_FP64_SWEEPS, -1, 0),
    (adg.OPT_FP64_SWEEPS, 65, 2),
    (adg.OPT_SCRATCH_BYTES, 0, 2 ** 30),
    (adg.OPT_SUBCELL_FP64_SWEEPS, 4, 3),
    (adg.OPT_FLUX, 2, 1),
    (adg.OPT_CFL, -0.1, 0.0),
    (adg.OPT_SLOT_CAPACITY, 0, 16),
    (adg.OPT_END_TIME, -1.0, 0.2),
])
def test_option_ranges_without_device_work(lib, key, bad, good):
    """Out-of-range option values are refused with ADG_ERR_ARG and a message;
    in-range values are taken (all before any device allocation)."""
    h = ctypes.c_void_p()
    g = adg.AdgGrid()
    g.dim = 2
    for k in range(3):
        g.n[k] = 4
        g.dx[k] = 0.25
    bcs = (ctypes.c_int * 6)(0, 0, 0, 0, 0, 0)
    assert lib.adg_create(ctypes.byref(g), 3, 1.4, bcs, adg.PREC_MIXED_FP32, ctypes.byref(h)) == 0
    try:
        assert lib.adg_set_option(h, key, float(bad)) == adg.ERR_ARG
        assert lib.adg_last_error(h)
        assert lib.adg_set_option(h, key, float(good)) == 0
    finally:
        lib.adg_destroy(h)


def test_predictor_shapes_that_do_not_apply_are_refused(lib):
    """ADG_OPT_PREDICTOR: the warp-per-cell shapes need mixed precision with
    no FP64 Picard sweep (2D N <= 5, 3D); both block widths apply everywhere."""
    f64 = adg.Solver(2, (4, 4), (0, 0), (0.1, 0.1), (0, 0, 0, 0), 5, prec=adg.PREC_FP64)
    mx5 = adg.Solver(2, (4, 4), (0, 0), (0.1, 0.1), (0, 0, 0, 0), 5, prec=adg.PREC_MIXED_FP32)
    mx7 = adg.Solver(2, (4, 4), (0, 0), (0.1, 0.1), (0, 0, 0, 0), 7, prec=adg.PREC_MIXED_FP32)
    for s, bad, good in ((f64, adg.PRED_WARP4, adg.PRED_BLOCK_ALT),
                         (mx5, 6, adg.PRED_WARP1),
                         (mx7, adg.PRED_WARP2, adg.PRED_BLOCK_ALT)):
        with pytest.raises(adg.AdgError) as e:
            s.set_option(adg.OPT_PREDICTOR, bad)
        assert e.value.code == adg.ERR_ARG
        s.set_option(adg.OPT_PREDICTOR, good)
        for v in (-1, -2):
            s.set_option(adg.OPT_PREDICTOR, v)
        with pytest.raises(adg.AdgError):
            s.set_option(adg.OPT_PREDICTOR, 6)
    # one FP64 sweep makes the N = 5 mixed state use the block kernel
    mx5.set_option(adg.OPT_FP64_SWEEPS, 1)
    with pytest.raises(adg.AdgError):
        mx5.set_option(adg.OPT_PREDICTOR, adg.PRED_WARP4)
    for s in (f64, mx5, mx7):
        s.close()


def test_tf32_precision_mode(lib):
    """ADG_PREC_MIXED_TF32 exists where the tensor-pipe predictor shape does
    (2D N <= 5, 3D) and is refused elsewhere."""
    s = adg.Solver(2, (4, 4), (0, 0), (0.1, 0.1), (0, 0, 0, 0), 5, prec=adg.PREC_MIXED_TF32)
    s.close()
    s = adg.Solver(3, (2, 2, 2), (0, 0, 0), (0.1,) * 3, (0,) * 6, 3, prec=adg.PREC_MIXED_TF32)
    s.close()
    with pytest.raises(adg.AdgError):
        adg.Solver(2, (4, 4), (0, 0), (0.1, 0.1), (0, 0, 0, 0), 6, prec=adg.PREC_MIXED_TF32)
