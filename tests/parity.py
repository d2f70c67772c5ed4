"""Element-by-element comparison of the CUDA path with the CPU oracle.

Tolerances (FP32 path against the float64 oracle):
  * state, observation features: |gpu - oracle| <= 1e-4 m + 1e-5 * |oracle|;
  * flags, rewards, done, index sets: identical, except decisions whose
    float64 margin is within 1e-5 m of the cutoff (zero penetration, goal
    radius, observation radius) and slots whose two candidates have float64
    distances within 1e-5 m of each other (tied rank).  Every exception is
    returned to the caller so that tests can report it.

Teacher forcing: the oracle always starts a step from the GPU's own state,
and decisions and observations are evaluated on the GPU's post-step state,
so FP32 rounding of earlier steps never accumulates into the comparison.
"""
from __future__ import annotations

import dataclasses

import numpy as np

ATOL = 1e-4
RTOL = 1e-5
TIE = 1e-5


def close(g, o):
    return np.abs(g.astype(np.float64) - o.astype(np.float64)) <= ATOL + RTOL * np.abs(o.astype(np.float64))


@dataclasses.dataclass
class Exceptions:
    items: list = dataclasses.field(default_factory=list)

    def add(self, *a):
        self.items.append(a)

    def __len__(self):
        return len(self.items)


def check_state(gpu_post, ora_post, active, ex: Exceptions, step=None):
    ok = close(gpu_post[active], ora_post[active])
    if not ok.all():
        bad = np.argwhere(~ok)
        i = np.nonzero(active)[0][bad[0, 0]]
        raise AssertionError(f"step {step}: state mismatch at agent {i}: gpu {gpu_post[i]} oracle {ora_post[i]}")


def check_decisions(g, o, ex: Exceptions, step=None):
    """g: dict(flags, reward, done, world_done) from the GPU; o: oracle step
    output with flags and margins (decisions on the GPU's post-step state)."""
    flags_g, flags_o = g["flags"], o["flags"]
    diff = np.nonzero(flags_g != flags_o)[0]
    for i in diff:
        x = int(flags_g[i]) ^ int(flags_o[i])
        ok = True
        if x & 4:
            ok &= abs(o["coll_margin"][i]) <= TIE
        if x & 8:
            ok &= abs(o["off_margin"][i]) <= TIE
        if x & 2:
            ok &= abs(o["goal_margin"][i]) <= TIE
        if x & 1:
            ok &= (abs(o["coll_margin"][i]) <= TIE or abs(o["off_margin"][i]) <= TIE or abs(o["goal_margin"][i]) <= TIE)
        if not ok:
            raise AssertionError(f"step {step}: flags differ at agent {i}: gpu {flags_g[i]:#x} oracle {flags_o[i]:#x} "
                                 f"margins coll {o['coll_margin'][i]} off {o['off_margin'][i]} goal {o['goal_margin'][i]}")
        ex.add("flag", step, int(i), int(flags_g[i]), int(flags_o[i]))
    same = np.ones(len(flags_g), bool)
    same[diff] = False
    np.testing.assert_array_equal(g["reward"][same], o["reward"][same], err_msg=f"reward, step {step}")
    np.testing.assert_array_equal(g["done"][same], o["done"][same], err_msg=f"done, step {step}")
    if len(diff) == 0:
        np.testing.assert_array_equal(g["world_done"], o["world_done"], err_msg=f"world_done, step {step}")


def _slots(gi, oi, gfeat, ofeat, fw, fetch, R, ex: Exceptions, tag, agent, step):
    """Compare one agent's slot list (indices gi / oi, features [n, fw])."""
    n = len(gi)
    eq = gi == oi
    if eq.all():
        ok = close(gfeat, ofeat)
        if not ok.all():
            r = int(np.argwhere(~ok)[0, 0])
            raise AssertionError(f"step {step} agent {agent} {tag} slot {r}: gpu {gfeat[r]} oracle {ofeat[r]}")
        return
    ok = close(gfeat[eq], ofeat[eq])
    if not ok.all():
        r = int(np.nonzero(eq)[0][np.argwhere(~ok)[0, 0]])
        raise AssertionError(f"step {step} agent {agent} {tag} slot {r}: gpu {gfeat[r]} oracle {ofeat[r]}")
    for r in np.nonzero(~eq)[0]:
        g, o = int(gi[r]), int(oi[r])
        dg = fetch(g)[1] if g >= 0 else None
        do = fetch(o)[1] if o >= 0 else None
        if dg is not None and do is not None:
            allowed = abs(dg - do) <= TIE
        elif dg is None:
            allowed = abs(do - R) <= TIE
        else:
            allowed = abs(dg - R) <= TIE
        if not allowed:
            raise AssertionError(f"step {step} agent {agent} {tag} slot {r}: gpu picked {g} (d={dg}), "
                                 f"oracle {o} (d={do})")
        exp = fetch(g)[0] if g >= 0 else np.zeros(fw, np.float32)
        if not close(gfeat[r], exp).all():
            raise AssertionError(f"step {step} agent {agent} {tag} slot {r} (tie exception): gpu {gfeat[r]} vs {exp}")
        ex.add(tag, step, agent, int(r), g, o, dg, do)


def check_obs(gobs, gri, gpi, oracle, oobs, ori, opi, K, P, R, ex: Exceptions, step=None, agents=None):
    A = gobs.shape[0]
    agents = range(A) if agents is None else agents
    for i in agents:
        ego_ok = close(gobs[i, :8], oobs[i, :8])
        if not ego_ok.all():
            raise AssertionError(f"step {step} agent {i} ego: gpu {gobs[i, :8]} oracle {oobs[i, :8]}")
        if P:
            gp = gobs[i, 8:8 + 8 * P].reshape(P, 8)
            op = oobs[i, 8:8 + 8 * P].reshape(P, 8)
            _slots(gpi[i], opi[i], gp, op, 8, lambda j, i=i: oracle.partner(i, j), R, ex, "partner", i, step)
        if K:
            gr = gobs[i, 8 + 8 * P:].reshape(K, 4)
            orr = oobs[i, 8 + 8 * P:].reshape(K, 4)
            _slots(gri[i], ori[i], gr, orr, 4, lambda j, i=i: oracle.road_point(i, j), R, ex, "road", i, step)
