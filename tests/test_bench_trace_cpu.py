"""CPU test of the bench's reading of the sweep kernel's timestamps (trace_summary):
a synthetic relaxation with known phase lengths, control steps and block placement."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _synthetic():
    # 3 sweeps of 4 tiles, 2 blocks (on SMs 0 and 1), each block runs two items per sweep
    # back to back: wait 0.5 us, copy 2 us, update 5 us, write-back 1 us; the sweep's
    # ticket 1.8 us after its last update, the control step 2.7 us after the ticket
    S, ntiles = 3, 4
    it = np.zeros((S, ntiles, 6), np.int64)
    ctl = np.zeros((4096, 2), np.int64)
    for s in range(S):
        base = 1_000 + s * 100_000
        for i in range(ntiles):
            t0 = base + (8_500 if i >= 2 else 0)
            t1 = t0 + 500
            t2 = t1 + 2_000
            t3 = t2 + 5_000
            it[s, i] = [t0, t1, t2, t3, t3 + 1_000, (i % 2) | ((i % 2) << 32)]
        last = base + 16_000
        ctl[17 + s] = [last + 1_800, last + 1_800 + 2_700]
    return it, ctl


def test_trace_summary_recovers_the_phase_lengths():
    import bench
    it, ctl = _synthetic()
    r = bench.trace_summary(it, ctl, True, 4)
    assert r["sweeps"] == 3 and r["items"] == 12 and r["blocks"] == 2
    assert r["us_wait"] == pytest.approx(0.5)
    assert r["us_copy"] == pytest.approx(2.0)
    assert r["us_update"] == pytest.approx(5.0)
    assert r["us_writeback"] == pytest.approx(1.0)
    assert r["us_per_sweep"] == pytest.approx(100.0)
    assert r["us_last_update_to_ticket"] == pytest.approx(1.8)
    assert r["us_control_step"] == pytest.approx(2.7)
    # next sweep's first copy lands 2.5 us after its start, 100 us after the previous start
    assert r["us_publish_to_first_copy_landed"] == pytest.approx(100.0 + 2.5 - 16.0 - 4.5)
    # 12 updates of 5 us over 2 blocks x (last update - first item taken)
    assert r["update_share_of_block_time"] == pytest.approx(60.0 / (2 * (216.0 + 1.0 - 1.0)))
    assert r["mid_sweep_tiles_per_sm"] == {"max": 2, "idle_sms": 2, "histogram": [2, 0, 2]}


def test_trace_summary_ignores_items_that_did_not_run():
    import bench
    it, ctl = _synthetic()
    it2 = np.concatenate([it, np.zeros((1, 4, 6), np.int64)])       # a sweep never started
    it2[0, 3] = 0                                                     # and one item of sweep 0
    r = bench.trace_summary(it2, ctl, False, 4)
    assert r["items"] == 11 and r["us_copy"] == pytest.approx(2.0)
    assert "us_control_step" not in r
