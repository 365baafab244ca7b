"""Host-side logic that needs no GPU: grouping views into frames by capacity (the batched
queue and training workloads size their frames with it) and the frame workspace sizing."""
import numpy as np

from paper_2404_01133_b300 import torch_api as ta


def test_waves_keep_order_and_respect_capacities():
    rng = np.random.default_rng(3)
    sel = rng.integers(1, 3_000_000, size=200).tolist()
    ent = rng.integers(1, 5_000_000, size=200).tolist()
    n_cap_max, k_cap_max = 40_000_000, 60_000_000
    groups = ta.waves(sel, ent, n_cap_max=n_cap_max, k_cap_max=k_cap_max)
    flat = [v for g in groups for v in g[0]]
    assert flat == list(range(200))                      # every view once, in order
    for views, n_cap, k_cap in groups:
        # the sizes cover every view of the group with the documented slack
        assert n_cap == sum(int(sel[v] * 1.05) + 1024 for v in views)
        assert k_cap == sum(int(ent[v] * 1.05) + 4096 for v in views)
        assert n_cap <= n_cap_max and k_cap <= k_cap_max
    # groups are maximal: the next view would not have fitted
    for (views, n_cap, k_cap), (nxt, _, _) in zip(groups, groups[1:]):
        v = nxt[0]
        s2, e2 = int(sel[v] * 1.05) + 1024, int(ent[v] * 1.05) + 4096
        assert n_cap + s2 > n_cap_max or k_cap + e2 > k_cap_max


def test_waves_oversized_view_gets_its_own_group():
    groups = ta.waves([10, 500, 10], [10, 10, 10], n_cap_max=300, k_cap_max=10_000)
    assert [g[0] for g in groups] == [[0], [1], [2]]
    assert ta.waves([], []) == []
