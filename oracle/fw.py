"""The limiting-amplitude ("full wave", FW) baseline (oracle).

Section 6: FW marches the time-domain DG scheme with the periodic source from
zero initial data, U^(l) = P_{psi,w} U^(l-1), U^(0) = 0, and after l simulated
periods takes the filtered field F_{psi,w} U^(l) (Section 2.1: the e^{i w t}
filter over one further period started from U^(l)).  By the limiting amplitude
principle (Section 1) F_{psi,w} U^(l) tends to the time-harmonic solution as
l grows, for problems whose transients decay (impedance boundary, no
trapping); CMCG reaches the same discrete limit, F_{psi,w} of the periodic
initial state.

Test infrastructure only.
"""
from __future__ import annotations

import numpy as np

from .filtering import filtered_sweep
from .timestep import Stepper


def fw_state(st: Stepper, j_re, j_im=None, periods: int = 1) -> np.ndarray:
    """U^(periods): `periods` source sweeps from rest."""
    U = np.zeros((st.geo.nt, 6, st.geo.nodes.shape[1]))
    for _ in range(periods):
        U = st.P_psi(U, j_re, j_im)
    return U


def fw_solve(st: Stepper, j_re, j_im=None, periods: int = 1) -> np.ndarray:
    """F_{psi,w} U^(periods): the FW result after `periods` simulated periods."""
    return filtered_sweep(st, fw_state(st, j_re, j_im, periods), j_re, j_im)
