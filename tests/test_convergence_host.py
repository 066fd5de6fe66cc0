"""Host logic of the time-to-steady rules (no GPU): a scripted stand-in for a
Lattice reports the inlet density that gives a chosen permeability at each
check, and the 0.1 % rule must report the first step of the first run of
`hold` consecutive checks within tolerance, restart the run on a miss, and
report failure when the budget ends first."""
import math

import pytest

from paper_1806_10589_gb300 import convergence as cv

TAU = 0.8
SHAPE = (21, 6, 5)
Q = 3e-3


def _rho_in(k):
    """Inverse of Darcy's law as convergence.permeability states it."""
    nz, ny, nx = SHAPE
    nu = cv.CS2 * (TAU - 0.5)
    return 1.0 + nu * (Q / (nx * ny)) * (nz - 1) / (cv.CS2 * k)


class ScriptedLattice:
    shape = SHAPE

    def __init__(self, ks, q_outs=None, every=100):
        self.ks, self.q_outs, self.every, self.t = ks, q_outs, every, 0

    def _check(self):
        return min(self.t // self.every, len(self.ks)) - 1

    def step(self, n):
        self.t += n

    def get_flux(self, face):
        c = self._check()
        if face == 4:
            return Q, _rho_in(self.ks[c])
        return (self.q_outs[c] if self.q_outs else Q), 1.0


def test_permeability_inverts():
    for k in (0.05, 1.0, 37.5):
        assert math.isclose(cv.permeability(Q, SHAPE, TAU, _rho_in(k), 1.0), k, rel_tol=1e-12)
    assert cv.permeability(Q, SHAPE, TAU, 1.0, 1.0) == float("inf")


def test_first_step_of_the_holding_run():
    # checks at steps 100, 200, ...: in at 300 and 400, out at 500, in from 600 on
    ks = [2.0, 1.2, 1.0005, 0.9995, 1.01, 1.0, 1.0009, 0.9991, 1.0, 1.0, 1.0]
    r = cv.run_to_reference(ScriptedLattice(ks), Q, TAU, 1.0, rtol=1e-3, hold=4, check_every=100)
    assert r["reached"] and r["steps"] == 600 and r["steps_run"] == 900


def test_budget_ends_before_the_rule_holds():
    ks = [1.0, 1.0, 1.002] * 10
    r = cv.run_to_reference(ScriptedLattice(ks), Q, TAU, 1.0, rtol=1e-3, hold=3, check_every=100,
                            max_steps=1500)
    assert not r["reached"] and r["steps"] is None and r["seconds"] is None and r["steps_run"] == 1500


@pytest.mark.parametrize("require", [False, True])
def test_outlet_flux_condition(require):
    ks = [1.0] * 8
    q_outs = [Q * 1.01] * 3 + [Q] * 5  # outlet flux settles at the fourth check
    r = cv.run_to_reference(ScriptedLattice(ks, q_outs), Q, TAU, 1.0, rtol=1e-3, hold=3, check_every=100,
                            require_q_out=require)
    assert r["steps"] == (400 if require else 100)
