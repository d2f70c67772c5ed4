"""Host-side logic of bench.py (no GPU): the active and controlled agent-step
counts on hand-made done traces, and the throughput arithmetic."""
import numpy as np

import bench


def test_active_agent_steps_hand_trace():
    # two worlds: [0, 1] and [2]; T = 4
    off = np.array([0, 2, 3])
    done = np.array([[0, 1, 0],      # after step 0: agent 1 done
                     [0, 1, 0],
                     [1, 1, 1],      # after step 2: everyone done -> both worlds restart
                     [0, 0, 0]], np.uint8)
    # step 0: 3 in; step 1: agent 1 out -> 2; step 2: 2; step 3: worlds ended -> all 3 back
    assert bench.active_agent_steps(done, off) == 3 + 2 + 2 + 3


def test_controlled_agent_steps_excludes_uncontrolled_agents():
    off = np.array([0, 3, 5])
    static = np.array([False, True, False, True, True])       # world 1 has no controlled agent
    done = np.array([[0, 1, 0, 1, 1],
                     [1, 1, 0, 1, 1],
                     [1, 1, 1, 1, 1],                        # world 0's controlled agents both done: restart
                     [0, 1, 0, 1, 1]], np.uint8)
    # controlled agents: 0 and 2; step 0: 2; step 1: 2; step 2: agent 0 out -> 1; step 3: restart -> 2
    assert bench.controlled_agent_steps(done, static, off) == 2 + 2 + 1 + 2
    # with nobody static it is the active count
    assert bench.controlled_agent_steps(done, np.zeros(5, bool), off) == bench.active_agent_steps(done, off)


def test_whole_job_rate_single_rank():
    t, rate = bench.whole_job_rate(1000, 250.0, 1, None)
    assert t == 250.0 and rate == 1000 / 0.25
