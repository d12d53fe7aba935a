"""Host logic of uneven batches (no GPU): the packing of x and phi that
group_layout produces for mck_group_create."""

import types

import numpy as np
import pytest

import paper_1702_08159_gb300 as mck


def _plans(ds):
    return [types.SimpleNamespace(d=d) for d in ds]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_layout_packs_without_overlap(seed):
    g = np.random.default_rng(seed)
    plans = _plans([64, 1024, 16384])
    n = 40
    pidx = g.integers(0, 3, n)
    E = g.integers(1, 33, n)
    d = np.array([plans[p].d for p in pidx])
    in_dim = np.array([g.integers(1, dd + 1) for dd in d])
    order = g.permutation(n)
    items, x_len, phi_len = mck.group_layout(plans, pidx, E, in_dim, order)
    assert x_len == int(((in_dim + 3) // 4 * 4).sum())
    assert phi_len == int((2 * E * d).sum())
    # every item's slots lie inside the arrays, phi offsets are 16-byte aligned,
    # x slots start on 4-float boundaries, and packing follows `order`
    assert np.all(items["phi_offset"] % 4 == 0) and np.all(items["x_offset"] % 4 == 0)
    assert np.all(items["x_offset"] + items["in_dim"] <= x_len)
    assert np.all(items["phi_offset"] + 2 * items["E"] * d <= phi_len)
    xo = items["x_offset"][order]
    po = items["phi_offset"][order]
    assert np.all(np.diff(xo) > 0) and np.all(np.diff(po) > 0)
    # no two items overlap in x or in phi
    xe = np.sort(np.stack([items["x_offset"], items["x_offset"] + items["in_dim"]], 1), 0)
    pe = np.sort(np.stack([items["phi_offset"], items["phi_offset"] + 2 * items["E"] * d], 1), 0)
    assert np.all(xe[1:, 0] >= xe[:-1, 1]) and np.all(pe[1:, 0] >= pe[:-1, 1])
    assert np.array_equal(items["plan"], pidx) and np.array_equal(items["E"], E)


def test_layout_default_order_and_empty():
    items, x_len, phi_len = mck.group_layout(_plans([32]), [0, 0], [1, 2], [3, 32])
    assert list(items["x_offset"]) == [0, 4] and x_len == 36
    assert list(items["phi_offset"]) == [0, 64] and phi_len == 64 + 128
    items, x_len, phi_len = mck.group_layout(_plans([32]), [], [], [])
    assert len(items) == 0 and x_len == 0 and phi_len == 0
