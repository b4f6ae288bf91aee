"""Worked numbers printed in the paper (tests/golden/paper_values.txt)."""
import math
import os

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def _load():
    vals = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, val = line.split()[:2]
        vals[key] = float(val)
    return vals


def test_wavenumbers_and_wavelengths():
    v = _load()
    for f in (200, 800, 1000):
        k = 2 * math.pi * f / 340.0
        assert abs(k - v["k_f%d_c340" % f]) < 5e-3
        assert abs(340.0 / f - v["lambda_f%d" % f]) < 1e-9


def test_storage_identities():
    """nnz(T) = nnz(S) = 2 L^2 N and 16 N^2 bytes for the dense matrix."""
    v = _load()
    assert 2 * 8 ** 2 * 4332 == v["nnzTS_N4332_L8"]
    assert 2 * 8 ** 2 * 8112 == v["nnzTS_N8112_L8"]
    assert abs(16 * 4332 ** 2 / 1e6 - v["dense_MB_N4332"]) < 1
    assert abs(16 * 8112 ** 2 / 1e6 - v["dense_MB_N8112"]) < 1
    assert abs(16 * 174298 ** 2 / 1e9 - v["dense_GB_N174298"]) < 1


def test_duct_amplitude():
    assert abs(1.3 * 340.0 - _load()["duct_abs_rho_c"]) < 1e-9
