"""Every branch of reaction resolution against the FP64 reference.

One reaction per species (closest pair first, lower ids breaking ties) is resolved on the
GPU by a conflict-free fast path plus rounds of locally-dominant selection, and the events
of a step are then ordered by (train, id_lo) for the product ids. The rounds run in shared
memory for up to 1,536 conflicting accepted pairs and in global memory beyond; the events
are ordered in shared memory for up to 8,192 events (a bucket sort, or a block radix sort
when the keys cluster) and in global memory beyond. The results must not depend on the
branch: each case here forces one branch, shows through the library's counters that it
ran, and requires event lists, per-step counts, tallies and positions identical to the
reference's. Runs through the C ABI on the GPU."""
import numpy as np
import pytest

from harness import assert_fp64_parity, cuda_available, gpu_batch_run, gpu_run, oracle_run
from paper_2509_03313_gb300 import chem, workloads as W

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")]


def _dense(n, L, seed, n_steps, dt=1e-9):
    counts = (W.MIX_COUNTS * n / W.MIX_COUNTS.sum()).astype(np.int64)
    p = W.uniform_mixture(counts, L, seed=seed)
    return W.Workload("dense", L, [p], W.Schedule(dt_min=dt, dt_max=dt), t_end=n_steps * dt)


def test_crowded_step_takes_the_global_memory_rounds_and_event_order():
    # 40,000 species in a 100 nm box (about 80 mM): in the first 1 ns step about 23,000
    # accepted pairs share a species with another and about 10,000 events commit.
    wl = _dense(40000, 100.0, seed=3, n_steps=2)
    g = gpu_run(wl, 3, capacity=80000)
    o = oracle_run(wl, 3)
    st = g["stats"]
    assert st["max_conflict_pairs"] > 1536 and st["react_rounds_global"] >= 1, st
    assert st["max_step_events"] > 8192 and st["react_order_global"] >= 1, st
    assert o.events_total.sum() > 8192
    assert_fp64_parity(g, o, wl.L)


def test_crowded_step_in_the_persistent_kernel():
    # The persistent kernel resolves every step in global memory.
    wl = _dense(12000, 80.0, seed=5, n_steps=3)
    g = gpu_run(wl, 5, capacity=24000, launch_mode=chem.CHEM_LAUNCH_PERSISTENT)
    o = oracle_run(wl, 5)
    st = g["stats"]
    assert st["react_rounds_global"] >= 1 and st["react_order_global"] >= 1, st
    assert o.events_total.sum() > 1000
    assert_fp64_parity(g, o, wl.L)


def test_clustered_event_keys_take_the_block_radix_order():
    # Two trains in one context: train 1's event keys carry its index in the top bit,
    # so train 0's events all fall into one bucket of the bucket sort, which then hands
    # the step to the block radix sort (shared memory, one kernel per phase).
    wls = [_dense(3000, 100.0, seed=7, n_steps=12), _dense(3000, 100.0, seed=8, n_steps=12)]
    stats = {}
    outs = gpu_batch_run(wls, [7, 8], [0, 1], launch_mode=chem.CHEM_LAUNCH_PHASES, stats=stats)
    assert stats["react_order_radix"] >= 1, stats
    for b, (wl, g) in enumerate(zip(wls, outs)):
        o = oracle_run(wl, 7 + b, train_id=b)
        assert o.events_total.sum() > 100
        assert_fp64_parity(g, o, wl.L)


def test_sparse_steps_stay_in_shared_memory():
    # The usual case: few conflicts and events per step never leave shared memory.
    wl = W.uniform_2000(seed=2, L=200.0, n_steps=60)
    g = gpu_run(wl, 2)
    st = g["stats"]
    assert st["react_rounds_global"] == 0 and st["react_order_global"] == 0, st
    assert st["max_step_events"] > 0
