"""Oracle for measurement trajectories and shadow snapshots (test infrastructure).

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's
CPU-baseline leg use this module.  It follows the definitions step by step with
the plain C routines of ``oracle/sv.c`` (unfused gates, single-qubit projective
measurements), in complex128.

* MIPT trajectory (Sec. VII.C): per time step, the step's two-qubit gates in
  order, then every selected qubit measured in the Z basis, in increasing qubit
  order, by the Born rule: outcome 0 iff u < p0 = P(qubit = 0) of the current
  state; the state is projected and renormalised; the trajectory's probability
  is the product of the outcome probabilities (returned as its natural log).
* Shadow snapshot (Sec. VII.A): the state rotated into the snapshot's Pauli
  basis, then every qubit measured in the Z basis the same way.
"""
from __future__ import annotations

import math

import numpy as np

from . import sv


def mipt_trajectory(n, gates, pools_t, masks_t, u_t, psi0=None):
    """One trajectory: ``pools_t[t]`` is the item's complex128 matrix pool of step t
    (gate matrices at their mat_off), ``masks_t[t]`` the measured-qubit bit mask,
    ``u_t[t][q]`` the Born uniforms.  Returns dict(psi, outcomes [D][n] (-1 where
    not measured), p0 [D][n] (nan where not measured), logp)."""
    D = len(pools_t)
    psi = sv.zero_state(n) if psi0 is None else np.array(psi0, dtype=np.complex128)
    outcomes = np.full((D, n), -1, dtype=np.int8)
    p0s = np.full((D, n), np.nan)
    logp = 0.0
    for t in range(D):
        pool = np.empty(2 * pools_t[t].size)
        pool[0::2] = pools_t[t].real
        pool[1::2] = pools_t[t].imag
        psi = sv.apply(n, gates, pool, None, psi=psi)
        for q in range(n):
            if (int(masks_t[t]) >> q) & 1:
                o, prob, p0 = sv.measure_qubit(n, psi, q, float(u_t[t][q]))
                outcomes[t, q] = o
                p0s[t, q] = p0
                logp += math.log(prob)
    return dict(psi=psi, outcomes=outcomes, p0=p0s, logp=logp)


def basis_change(n, bases):
    """Gate list taking the Pauli basis of each qubit to Z: H for X (bases 1),
    H S^dagger for Y (bases 2), nothing for Z (bases 3).  (The CUDA path uses
    RY(-pi/2) and RX(pi/2), which differ from these by diagonal phases only, so
    every measurement probability is the same.)"""
    from workloads import Circuit
    c = Circuit(n)
    sdg = np.diag([1.0, -1j])
    for q, b in enumerate(bases):
        if b == 1:
            c.h(q)
        elif b == 2:
            c.unitary((q,), sdg)
            c.h(q)
    return c.to_ir()


def shadow_snapshot(n, psi, bases, u):
    """Rotate ``psi`` into the snapshot's bases and measure every qubit (increasing
    order, Born rule with ``u[q]``).  Returns (outcomes [n], p0 [n], final state)."""
    g, p = basis_change(n, bases)
    phi = sv.apply(n, g, p, None, psi=psi)
    out = np.zeros(n, dtype=np.int8)
    p0s = np.zeros(n)
    for q in range(n):
        o, _, p0 = sv.measure_qubit(n, phi, q, float(u[q]))
        out[q] = o
        p0s[q] = p0
    return out, p0s, phi
