"""GPU: the arithmetic-pipe probe (adg_pipe_rates) and the Newton-Raphson
reciprocal the mixed-precision path uses for 1 / rho in its FP64 terms:
within one unit in the last place of CUDA's 1.0 / x on 2^22 hashed values
spanning 2^-60 .. 2^60, both signs."""
import pytest

from paper_1406_7416_gb300 import adg, build_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib.build()
    adg.load_library()


def test_pipe_rates_and_newton_reciprocal():
    r = adg.pipe_rates()
    for key in ("dfma", "ffma", "f64_to_f32", "f64_compare", "f64_reciprocal_div",
                "f64_reciprocal_newton"):
        assert r[key] > 0.0, key
    assert r["ffma"] > 10 * r["dfma"]            # the FP32 pipe is far wider than the FP64 pipe
    assert r["newton_max_ulp"] <= 1.0
    assert 0.0 <= r["newton_differ_fraction"] < 0.5
    print(r)
