"""How far two oracle runs of Algorithm 1 drift apart when only the rounding
order of one step differs: the second run takes its POD (Eq. pod) from the
thin SVD of the window with its rows in reverse order, which is the same
mathematics with other rounding.  The hybrid map amplifies such differences
(measured on the 64^2 oblique shock with k = 3: about 4x per hybrid step once
the basis tracks the front), so an FP64 GPU trajectory, whose every stage
matches the oracle to 1e-12 on identical inputs, drifts from the oracle at
the same rate.  The lockstep tests bound the GPU's drift by this spread.
Test infrastructure: it calls only oracle/ and workloads.py."""
import numpy as np

from oracle import arom, rom


def _pod_rows_reversed(pod):
    def pod_rev(Xc, m, pod_tol, abs_floor=0.0):
        Phi, s = pod(np.ascontiguousarray(Xc[::-1]), m, pod_tol, abs_floor)
        Phi = np.ascontiguousarray(Phi[::-1])
        for j in range(Phi.shape[1]):        # the oracle's sign rule
            i = int(np.argmax(np.abs(Phi[:, j])))
            if Phi[i, j] < 0.0:
                Phi[:, j] = -Phi[:, j]
        return Phi, s
    return pod_rev


def rel_max(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def spread(q0, cfg, steps, ref_states):
    """Per-step relative max difference between the oracle run whose states
    are ref_states (one flat array per step) and the same run with the POD
    rows reversed."""
    pod = rom.pod
    rom.pod = _pod_rows_reversed(pod)
    try:
        B = arom.Arom(q0, cfg)
        out = []
        for k in range(steps):
            B.step()
            out.append(rel_max(B.gamma.reshape(-1), ref_states[k]))
    finally:
        rom.pod = pod
    return out


def newton_spread(q0, cfg, steps, ref_states, tighter=100.0):
    """Per-step relative max difference between the run of ref_states and the
    same run with every Newton solve taken `tighter` times further: how far
    apart two runs can lie that both stop their solves within the
    tolerance, after the method has carried the difference along."""
    B = arom.Arom(q0, cfg.with_(newton_tol=cfg.newton_tol / tighter))
    out = []
    for k in range(steps):
        B.step()
        out.append(rel_max(B.gamma.reshape(-1), ref_states[k]))
    return out


def bar(spread_k, floor=1e-12, factor=100.0):
    """The lockstep bound at one step: 1e-12 relative (the per-stage FP64
    tolerance) while the rounding-order spread is small, and 100x the spread
    once the method has amplified it beyond that (the GPU's own rounding
    differences start about 30-40x larger than a row reversal's)."""
    return max(floor, factor * spread_k)
