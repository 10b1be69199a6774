"""Batched PLE: every table configuration of the persistent kernel, the
autotuner that picks one per size class, and the CUDA-graph plan that
replays one batch layout.  All results bit-exact against the oracle."""
import numpy as np
import pytest

import gf2inputs as gi
from tests.gpu_util import to_dev, to_host, vec_dev
from tests.test_gpu_parity import _batched_check, make, ref_ple_1, assert_ple_equal

pytestmark = pytest.mark.gpu


def _mixed():
    """Matrices across all six size classes, with ragged widths and edges."""
    mats = []
    sizes = [(65, 70), (128, 128), (200, 130), (256, 250), (300, 500), (512, 512), (700, 1000),
             (1024, 1024), (1500, 1100), (2048, 900), (3000, 2500), (4096, 4096), (1, 1), (64, 1),
             (1, 200), (129, 4096), (4096, 65)]
    for k, (m, n) in enumerate(sizes):
        kind = ["dense", "sparse", "lowrank", "lastrow_pivot"][k % 4]
        mats.append((make(kind, m, n, 100 + k), m, n, k % 2))
    return mats


@pytest.fixture(scope="module")
def h():
    import paper_1111_6549_gb300 as g
    return g.Handle()


@pytest.mark.parametrize("config", range(5))
def test_every_batched_configuration_matches_oracle(h, config):
    h.batched_config(-1, config)
    try:
        assert h.batched_get_config() == [config] * 6
        _batched_check(h, _mixed())
        specs = gi.batch_recipe(count=200)
        _batched_check(h, [(gi.batch_matrix(sp), sp["m"], sp["n"], 0) for sp in specs])
    finally:
        h.batched_config(-1, -1)


def test_per_class_configurations_mixed_in_one_launch(h):
    for c, cfg in enumerate([2, 4, 1, 3, 0, 2]):
        h.batched_config(c, cfg)
    try:
        assert h.batched_get_config() == [2, 4, 1, 3, 0, 2]
        _batched_check(h, _mixed())
    finally:
        h.batched_config(-1, -1)


def test_autotune_picks_valid_configs_and_keeps_results(h):
    import paper_1111_6549_gb300 as g
    chosen, table = h.batched_autotune(reps=1)
    assert len(chosen) == g.BATCH_CLASSES and all(0 <= c < g.BATCH_CONFIGS for c in chosen)
    for c in range(g.BATCH_CLASSES):
        assert all(0 < t < 1e4 for t in table[c])
        assert table[c][chosen[c]] == min(table[c])
    _batched_check(h, _mixed())
    h.batched_config(-1, -1)


def test_bad_config_arguments(h):
    import paper_1111_6549_gb300 as g
    for cls, cfg in [(6, 0), (-2, 0), (0, 5), (0, -2)]:
        with pytest.raises(g.GF2Error):
            h.batched_config(cls, cfg)


def test_graph_plan_replays_match_oracle(h):
    import torch
    specs = gi.batch_recipe(count=300)
    mats = [gi.batch_matrix(sp) for sp in specs]
    dA = [to_dev(A) for A in mats]
    pristine = [a.clone() for a in dA]
    items = [(a, sp["m"], sp["n"], vec_dev(sp["m"]), vec_dev(min(sp["m"], sp["n"])), vec_dev(1))
             for a, sp in zip(dA, specs)]
    plan = h.batched_plan(items)
    try:
        for rep in range(2):
            for a, p in zip(dA, pristine):
                a.copy_(p)
            plan.launch()
            torch.cuda.synchronize()
            for (a, m, n, P, Q, rk), A in zip(items, mats):
                want = ref_ple_1(A, m, n)
                got = (int(rk.cpu()[0]), to_host(a, gi.words_for(n)), P.cpu().numpy()[:m],
                       Q.cpu().numpy()[:min(m, n)])
                assert_ple_equal(got, want)
            for _, _, _, P, Q, rk in items:
                P.fill_(-7)
                Q.fill_(-7)
                rk.fill_(-7)
    finally:
        plan.close()


def test_graph_plan_rejects_large_or_empty(h):
    import paper_1111_6549_gb300 as g
    big = to_dev(make("dense", 5000, 100, 1))
    with pytest.raises(g.GF2Error):
        h.batched_plan([(big, 5000, 100, vec_dev(5000), vec_dev(100), vec_dev(1))])
    with pytest.raises(g.GF2Error):
        h.batched_plan([])
