"""The in-graph loop: each level's iterations run inside a conditional WHILE
node whose body is one iteration, and the norm kernel leaves the loop when the
call's iteration budget is spent or the stop rule of Sec. 2.3 fires.

Checked against the two other schedules of the same kernels (the n-iteration
unrolled graph, test switch DISC_SW_UNROLLED_GRAPH, and plain stream launches,
DISC_SW_NO_GRAPH): bitwise the same field, the same iteration counts and norm
history, in one call or in chunks; and a stopped level costs no more kernels.
"""
import time

import numpy as np
import pytest

from paper_1204_6295_b300 import phantom

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def disc():
    from paper_1204_6295_b300 import disc as d
    return d


MODES = {"loop": 0, "unrolled": 8, "stream": 4}   # disc_set_test_switches bits


def _run(disc, mode, pair, chunks, **kw):
    with disc.test_switches(MODES[mode]):
        reg = disc.Registration(**kw)
    with reg:
        reg.set_images(pair.ct, pair.cbct)
        done = []
        for n in chunks:
            done.append(reg.iterate(n)[0])
        hist = [reg.norm_history(l) for l in range(kw["levels"])]
        return reg.get_field(), done, hist


@pytest.mark.parametrize("chunks", [(-1,), (7, 5, 30, -1)])
def test_loop_graph_matches_unrolled_and_stream(disc, chunks):
    pair = phantom.ellipsoid_pair(48, 40, 24, seed=21)
    kw = dict(patch=(5, 5, 5), sigma=1.0, levels=2, iters=(40, 200), stop_eps=2e-3)
    out = {m: _run(disc, m, pair, chunks, **kw) for m in MODES}
    f0, d0, h0 = out["loop"]
    assert sum(d0) < 240                             # the stop rule ended the fine level early
    for m in ("unrolled", "stream"):
        f, d, h = out[m]
        np.testing.assert_array_equal(f, f0)
        assert d == d0
        for a, b in zip(h, h0):
            np.testing.assert_array_equal(a, b)


def test_stopped_level_costs_no_kernels(disc):
    import torch
    pair = phantom.ellipsoid_pair(32, 32, 16, seed=8)
    kw = dict(patch=(3, 3, 3), sigma=1.0, levels=1, iters=(3000,), stop_eps=1e-2)
    times = {}
    for mode in ("loop", "unrolled"):
        with disc.test_switches(MODES[mode]):
            reg = disc.Registration(**kw)
        with reg:
            reg.set_images(pair.ct, pair.cbct)
            zero = np.zeros((3, 16, 32, 32), np.float32)
            reg.iterate(-1)                          # builds the graph
            reg.set_field(0, zero)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            done, _ = reg.iterate(-1)
            times[mode] = time.perf_counter() - t0
            assert 10 < done < 3000
    # the unrolled graph still launches every one of the 3000 iterations' kernels
    assert times["loop"] < 0.5 * times["unrolled"]


@pytest.mark.parametrize("fill_passes", [32, 3])
def test_masked_fill_loop_matches_stream(disc, fill_passes):
    """The masked form's fill passes: inside a captured graph they are the body of
    their own WHILE node (nested in the level's loop when the stop rule is on),
    with the pass index on the device; with plain stream launches the host queues
    every pass.  The fields, iteration counts and norm histories are bitwise the
    same, with every masked voxel reached (32 passes) or with a pass cap that
    leaves some unfilled (3)."""
    pair = phantom.ellipsoid_pair(48, 40, 24, seed=23)
    kw = dict(patch=(5, 5, 5), sigma=1.0, levels=2, iters=(12, 60), stop_eps=2e-3, mask_mode=1,
              fill_passes=fill_passes)
    out = {m: _run(disc, m, pair, (5, -1), **kw) for m in MODES}
    f0, d0, h0 = out["stream"]
    assert np.isfinite(f0).all() and np.abs(f0).max() > 0
    for m in ("loop", "unrolled"):
        f, d, h = out[m]
        np.testing.assert_array_equal(f, f0)
        assert d == d0
        for a, b in zip(h, h0):
            np.testing.assert_array_equal(a, b)
