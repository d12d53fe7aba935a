"""Uneven batches in one persistent launch (mck_group_*) against the oracle."""

import json

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import fastfood as ff

pytestmark = pytest.mark.gpu


def _oracle_item(plan, T, x, E):
    Te = {k: (v[:E] if isinstance(v, np.ndarray) else v) for k, v in T.items()}
    return ff.features(x[None].astype(np.float64), Te)[0]


def _scaled(x):
    return (x * np.float32(6.0 / np.sqrt(len(x)))).astype(np.float32)


@pytest.fixture(scope="module")
def mixed(mck, dev):
    """46 vectors, d = 2^6..2^14, E = 1..6 (<= 2 for d >= 2^12), RBF and Matern (d <= 256)."""
    rng = np.random.default_rng(7)
    Ls = list(range(6, 15))
    plans, keys = [], {}
    spec = []
    for i in range(46):
        L = int(Ls[i % len(Ls)])
        d = 1 << L
        kern = "matern" if (d <= 256 and i % 2) else "rbf"
        if (d, kern) not in keys:
            keys[(d, kern)] = len(plans)
            plans.append(mck.Plan(d, 6, kern, 1.0, 42, matern_t=40))
        E = int(rng.integers(1, 3 if L >= 12 else 7))
        in_dim = d - int(rng.integers(0, 4)) if i % 3 else d
        spec.append((keys[(d, kern)], E, in_dim))
    pidx = [s[0] for s in spec]
    items, x_len, phi_len = mck.group_layout(plans, pidx, [s[1] for s in spec], [s[2] for s in spec])
    xh = np.zeros(x_len, np.float32)
    xs = []
    for i, (p, E, in_dim) in enumerate(spec):
        v = _scaled(wl.gaussian(1, in_dim, seed=100 + i)[0])
        xh[items["x_offset"][i]: items["x_offset"][i] + in_dim] = v
        xs.append(v)
    tables = {}
    for (d, kern), p in keys.items():
        tables[p] = ff.plan_tables(d, 6, ff.RBF if kern == "rbf" else ff.MATERN, 1.0, t=40, seed=42)
    return plans, spec, items, x_len, phi_len, xh, xs, tables


def test_grouped_matches_oracle(mck, dev, mixed):
    plans, spec, items, x_len, phi_len, xh, xs, tables = mixed
    group = mck.Group(plans, items, x_len, phi_len)
    x = torch.from_numpy(xh).to(dev)
    phi = torch.full((phi_len,), float("nan"), device=dev)
    group.features(x, phi)
    out = phi.cpu().numpy()
    for i, (p, E, in_dim) in enumerate(spec):
        d = plans[p].d
        got = out[items["phi_offset"][i]: items["phi_offset"][i] + 2 * E * d]
        ref = _oracle_item(plans[p], tables[p], xs[i], E)
        assert np.abs(got - ref).max() <= 1e-5, (i, d, E)


@pytest.mark.parametrize("grain", [1, 3, 16])
def test_grouped_grains_agree(mck, dev, mixed, grain):
    plans, spec, items, x_len, phi_len, xh, xs, tables = mixed
    x = torch.from_numpy(xh).to(dev)
    a = mck.Group(plans, items, x_len, phi_len, grain=1).features(x, torch.zeros(phi_len, device=dev))
    g = mck.Group(plans, items, x_len, phi_len, grain=grain)
    b = g.features(x, torch.zeros(phi_len, device=dev))
    assert torch.equal(a, b)
    assert g.info()["grain"] == grain


def test_grouped_matches_batched_kernel(mck, dev):
    # Large-d Matern (too slow for the oracle at this size) against the batched
    # feature kernel, which the oracle pins at smaller sizes.
    for d in (1024, 4096):
        plan = mck.Plan(d, 4, "matern", 1.0, 5, matern_t=40)
        n = 10
        x = np.stack([_scaled(v) for v in wl.gaussian(n, d, seed=d)])
        E = [1 + i % 4 for i in range(n)]
        items, x_len, phi_len = mck.group_layout([plan], [0] * n, E, [d] * n)
        xh = np.zeros(x_len, np.float32)
        for i in range(n):
            xh[items["x_offset"][i]: items["x_offset"][i] + d] = x[i]
        phi = mck.Group([plan], items, x_len, phi_len).features(
            torch.from_numpy(xh).to(dev), torch.zeros(phi_len, device=dev)).cpu().numpy()
        full = mck.features(plan, torch.from_numpy(x).to(dev)).cpu().numpy()
        for i in range(n):
            o = items["phi_offset"][i]
            np.testing.assert_allclose(phi[o: o + 2 * E[i] * d], full[i, : 2 * E[i] * d], atol=1e-6)


def test_cuda_graph_replay(mck, dev, mixed):
    plans, spec, items, x_len, phi_len, xh, xs, tables = mixed
    g = mck.Group(plans, items, x_len, phi_len)
    x = torch.from_numpy(xh).to(dev)
    direct = g.features(x, torch.zeros(phi_len, device=dev)).clone()
    phi = torch.zeros(phi_len, device=dev)
    cap = mck.CapturedGroup(g, x, phi)
    phi.zero_()
    cap.replay()
    torch.cuda.synchronize()
    assert torch.equal(phi, direct)


def test_autotuner_and_cache(mck, dev, mixed, tmp_path):
    from paper_1702_08159_gb300.tune import tune_grain

    plans, spec, items, x_len, phi_len, xh, xs, tables = mixed
    g = mck.Group(plans, items, x_len, phi_len)
    x = torch.from_numpy(xh).to(dev)
    phi = torch.zeros(phi_len, device=dev)
    cache = str(tmp_path / "tune.json")
    best, times = tune_grain(g, x, phi, grains=(1, 2, 4), reps=2, cache=cache)
    assert best in (1, 2, 4) and set(times) == {1, 2, 4}
    assert g.info()["grain"] == best
    data = json.load(open(cache))
    assert len(data) == 1 and list(data.values())[0]["grain"] == best
    g2 = mck.Group(plans, items, x_len, phi_len)
    best2, _ = tune_grain(g2, x, phi, grains=(1, 2, 4), cache=cache)  # from the cache
    assert best2 == best and g2.info()["grain"] == best


def test_group_validation(mck, dev):
    plan = mck.Plan(256, 2, "rbf", 1.0, 1)
    with pytest.raises(mck.MckError):
        mck.Group([plan], [(1, 1, 256, 0, 0)], 256, 4096)      # plan index
    with pytest.raises(mck.MckError):
        mck.Group([plan], [(0, 3, 256, 0, 0)], 256, 4096)      # E > plan E
    with pytest.raises(mck.MckError):
        mck.Group([plan], [(0, 1, 256, 100, 0)], 256, 4096)    # x slot past x_len
    with pytest.raises(mck.MckError):
        mck.Group([plan], [(0, 2, 256, 0, 8)], 256, 1024)      # phi slot past phi_len
    with pytest.raises(mck.MckError, match="UNSUPPORTED"):
        mck.Group([mck.Plan(1 << 15, 1, "rbf", 1.0, 1)], [], 0, 0)
    g = mck.Group([plan], [], 0, 0)                             # empty batch
    g.features(torch.zeros(4, device=dev), torch.zeros(4, device=dev))
    g = mck.Group([plan], [(0, 1, 256, 0, 0)], 256, 512)
    with pytest.raises((ValueError, mck.MckError)):             # phi array too small
        g.features(torch.zeros(256, device=dev), torch.zeros(8, device=dev))
