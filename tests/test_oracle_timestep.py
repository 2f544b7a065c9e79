"""Pin of the CFL time step (Sec. III.B, DG time step with c/D = 0.4186)
against the time steps printed in Table I."""
import os

import ffe_workloads as W
from oracle.problem import Problem

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1_dt.txt")


def test_table1_time_steps():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for name, length, dt in rows:
        L = float(length)
        cfg = W.fast_wave()
        cfg["lo"], cfg["hi"] = (0.0, -0.1, -0.1), (L, 0.1, 0.1)
        cfg["n"] = (32, 1, 1)
        cfg["params"]["cfl"] = 0.3
        pr = Problem(cfg)
        # the table prints three significant digits
        assert abs(pr.dt - float(dt)) <= 0.006 * float(dt), (name, pr.dt, dt)
