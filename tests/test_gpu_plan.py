"""GPU plan tables against the oracle: B and Pi bit-exact, G and C within float32 rounding."""

import numpy as np
import pytest

from oracle import fastfood as ff

pytestmark = pytest.mark.gpu


def _bits_to_signs(bits, d):
    k = np.arange(d)
    return np.where((bits[:, k // 32] >> (k % 32)) & 1, -1.0, 1.0)


@pytest.mark.parametrize("d,E,seed", [(2, 1, 0), (16, 3, 42), (1024, 4, 42), (1024, 2, 0xFEEDFACECAFEBEEF),
                                      (4096, 2, 7), (1 << 15, 1, 3)])
def test_rbf_tables(mck, d, E, seed):
    sigma = 1.7
    plan = mck.Plan(d, E, "rbf", sigma, seed)
    t = plan.tables()
    ref = ff.plan_tables(d, E, ff.RBF, sigma, seed=seed)
    np.testing.assert_array_equal(_bits_to_signs(t["B_bits"], d), ref["B"])
    np.testing.assert_array_equal(t["perm"].astype(np.int64), ref["perm"])
    # G: float64 Box-Muller on both sides, rounded to float32 once here.
    g32 = ref["G"].astype(np.float32)
    ulp = np.spacing(np.abs(g32))
    assert np.all(np.abs(t["G"].astype(np.float64) - ref["G"]) <= ulp)
    assert np.mean(t["G"] == g32) > 0.999
    c32 = ref["Cs"].astype(np.float32)
    assert np.all(np.abs(t["Cs"].astype(np.float64) - ref["Cs"]) <= np.spacing(np.abs(c32)))
    plan.close()


@pytest.mark.parametrize("d,E,seed", [(2, 3, 0), (16, 3, 42), (1024, 4, 42), (4096, 2, 11)])
def test_laplace_tables(mck, d, E, seed):
    """Laplacian calibration: the chi_d radius over |N(0,1)|, float64 on both
    sides and rounded to float32 once."""
    sigma = 0.8
    plan = mck.Plan(d, E, "laplace", sigma, seed)
    t = plan.tables()
    ref = ff.plan_tables(d, E, ff.LAPLACE, sigma, seed=seed)
    np.testing.assert_array_equal(t["perm"].astype(np.int64), ref["perm"])
    c32 = ref["Cs"].astype(np.float32)
    assert np.all(t["Cs"] > 0)
    assert np.all(np.abs(t["Cs"].astype(np.float64) - ref["Cs"]) <= np.spacing(np.abs(c32)))
    assert "laplace" in repr(plan)
    plan.close()


@pytest.mark.parametrize("d,E,t", [(2, 2, 3), (64, 2, 40), (256, 1, 40), (1024, 1, 40)])
def test_matern_tables(mck, d, E, t):
    sigma = 1.0
    plan = mck.Plan(d, E, "matern", sigma, 42, matern_t=t)
    tab = plan.tables()
    ref = ff.plan_tables(d, E, ff.MATERN, sigma, t=t, seed=42) if d <= 256 else None
    if ref is not None:
        np.testing.assert_array_equal(tab["perm"].astype(np.int64), ref["perm"])
        np.testing.assert_allclose(tab["Cs"], ref["Cs"], rtol=2e-6, atol=0)
    else:
        # full-size: radii of a sample of rows (the oracle's literal sampler per row)
        ks = [0, 1, 17, 511, d - 1]
        r = ff.table_radius(d, E, ff.MATERN, t, seed=42, ks=ks)
        G = ff.table_G(d, E, seed=42)
        expect = r / np.linalg.norm(G, axis=1, keepdims=True) / (sigma * np.sqrt(d))
        np.testing.assert_allclose(tab["Cs"][:, ks], expect, rtol=2e-6, atol=0)
    plan.close()


@pytest.mark.parametrize("d,E", [(1 << 11, 32), (1 << 13, 4), (1 << 14, 32), (1 << 15, 2)])
def test_matern_tables_large_d(mck, d, E):
    """Matern calibration above d = 1024 (the uneven batch builds t = 40
    plans up to 2^14 with 32 expansions): sampled entries (e, k) against the
    oracle's literal ball sum (t d normals per entry), the radius over
    ||G_e|| and sigma sqrt d; float32 ball coordinates bound the agreement
    to 2e-6 relative."""
    sigma, t, seed = 1.0, 40, 42
    plan = mck.Plan(d, E, "matern", sigma, seed, matern_t=t)
    tab = plan.tables()
    plan.close()
    es = sorted({0, E // 2, E - 1})
    ks = sorted({0, 1, 511, d // 2 + 3, d - 1} | set(np.random.default_rng(d).integers(0, d, 2).tolist()))
    G = ff.table_G(d, E, seed=seed)
    r = ff.table_radius(d, E, ff.MATERN, t, seed=seed, ks=ks)
    expect = r / np.linalg.norm(G, axis=1, keepdims=True) / (sigma * np.sqrt(d))
    np.testing.assert_allclose(tab["Cs"][np.ix_(es, ks)], expect[es], rtol=2e-6, atol=0)
    assert np.all(tab["Cs"] > 0) and np.isfinite(tab["Cs"]).all()


def test_seed_determinism_and_independence(mck):
    a = mck.Plan(256, 2, "rbf", 1.0, 99).tables()
    b = mck.Plan(256, 2, "rbf", 1.0, 99).tables()
    c = mck.Plan(256, 2, "rbf", 1.0, 100).tables()
    for k in a:
        np.testing.assert_array_equal(a[k], b[k])
    assert not np.array_equal(a["perm"], c["perm"])


def test_plan_info_roundtrip(mck):
    import ctypes

    from paper_1702_08159_gb300 import _lib

    plan = mck.Plan(128, 5, "matern", 2.5, 1 << 40, matern_t=7)
    d, E, k, s, t, seed, dv = (ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double(),
                               ctypes.c_int32(), ctypes.c_uint64(), ctypes.c_int32())
    _lib.check(_lib.load().mck_plan_info(plan.handle, *(ctypes.byref(v) for v in (d, E, k, s, t, seed, dv))),
               "info")
    assert (d.value, E.value, k.value, s.value, t.value, seed.value, dv.value) == (128, 5, 1, 2.5, 7, 1 << 40, 0)
