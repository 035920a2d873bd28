"""Tip-steering (the paper's supplement): an actuator that acts only on the
tip and moves up as the tip grows.  The robot grows with the tip actuator
unpressurised; to steer, growth is stunted (the distal length is held fixed)
and the tip actuator, moved over the last `span` links, is pressurised; each
steering step re-solves the equilibrium at the present links
(``vine_relax`` with fix_length = 1).  The actuator update is
``vine_set_actuators``; every solve runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np


class TipSteering:
    """Drives a batch whose robots each carry one tip actuator.

    tip_act[i] is the index (in the scene's actuator order) of robot i's tip
    actuator; the other actuators keep their spans and pressures."""

    def __init__(self, batch, scene: dict, tip_act, span: int = 4):
        self.b = batch
        self.span = int(span)
        self.tip = np.asarray(tip_act, np.int64)
        self.pressure = np.asarray(scene["act_pressure"], np.float32).copy()
        self.begin = np.asarray(scene["act_begin"], np.float32).copy()
        self.end = np.asarray(scene["act_end"], np.float32).copy()
        self.pressure[self.tip] = 0.0
        self._push()

    def _push(self):
        self.b.set_actuators(self.pressure, self.begin, self.end)

    def spans(self, n_present):
        """The tip actuators' spans over the last `span` present links."""
        N = np.asarray(n_present, np.int64)
        end = np.maximum(N, 1).astype(np.float32)
        begin = np.maximum(end - self.span, 0.0).astype(np.float32)
        return begin, end

    def grow(self, n_steps: int):
        """Growth with the tip actuators unpressurised."""
        self.pressure[self.tip] = 0.0
        self._push()
        self.b.grow_step(int(n_steps))

    def steer(self, pressure):
        """One steering step: tip actuators over the last links at `pressure`
        (Pa, scalar or per robot), distal length held, equilibrium re-solved."""
        N = self.b.state()["N"]
        bgn, end = self.spans(N)
        self.begin[self.tip] = bgn
        self.end[self.tip] = end
        self.pressure[self.tip] = np.broadcast_to(np.asarray(pressure, np.float32), self.tip.shape)
        self._push()
        self.b.relax(fix_length=True)
