"""Host-side helpers of the benchmark (no GPU): the sampled schedule steps,
the oracle leg's stored states and error summaries, and the command line."""
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_timed_steps_spread_over_the_schedule():
    # step (i + 1/2) total / K, one per equal share of the schedule
    assert bench.timed_indices(2000, 20) == list(range(50, 2000, 100))
    assert bench.timed_indices(2000, 1) == [1000]
    assert bench.timed_indices(10, 10) == list(range(10))
    assert bench.timed_indices(10, 50) == list(range(10))
    idx = bench.timed_indices(2000, 7)
    assert len(idx) == 7 and idx == sorted(set(idx)) and 0 <= idx[0] and idx[-1] < 2000


def test_max_known_skips_missing_errors():
    # gamma errors are compared only where the constraint sets agree
    assert bench._max_known([None, 2.0e-6, 5.0e-7]) == 2.0e-6
    assert bench._max_known([None, None]) is None
    assert bench._max_known([]) is None


def test_subset_states_are_the_oracle_snapshots_of_the_scene():
    sc, states = bench.subset_states()
    assert sc.n == bench.SUBSET_BODIES
    steps = [k for k, *_ in states]
    assert steps[0] == 0 and steps == sorted(steps) and len(steps) >= 6
    vol = sc.meta["volume"]
    phis = [vol / float(np.prod(box)) for _, _, _, box in states]
    assert abs(phis[0] - 0.1) < 1e-6 and all(a < b for a, b in zip(phis, phis[1:])) and phis[-1] < 0.56
    for _, x, q, box in states:
        assert x.shape == (sc.n, 3) and q.shape == (sc.n, 4)
        assert np.allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-12)


def test_command_line_lists_every_leg():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True, text=True,
                       timeout=120, cwd=ROOT)
    assert r.returncode == 0
    for flag in ("--steps", "--warmup", "--gpus", "--impl", "--augmentation", "--only-augmentation",
                 "--only-colony", "--only-refinement", "--only-batched", "--only-learned", "--subset-steps"):
        assert flag in r.stdout, flag
