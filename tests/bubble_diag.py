"""Diagnostics of the two-dimensional bubble cases (test helper): extremes of
theta' = theta_l - 300 K and of the velocities, the density current's front
(the farthest node right of the axis where theta' < -1 K at the lowest
level), and the warm bubble's theta'-weighted centroid and top (theta' > 0.1
K).  Measurement only: none of the method's arithmetic."""
import numpy as np


def bubble_diagnostics(case, theta_l, u, w) -> dict:
    tp = np.asarray(theta_l, dtype=np.float64) - 300.0
    u = np.asarray(u, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    x = (np.arange(case.nx) + 0.5) * case.dx - case.init_args["xc"]
    z = (np.arange(case.nz) + 0.5) * case.dz
    out = {"theta_min": float(tp.min()), "theta_max": float(tp.max()), "w_min": float(w.min()),
           "w_max": float(w.max()), "u_absmax": float(np.abs(u).max())}
    cold = np.where((tp[0, 0] < -1.0) & (x > 0))[0]
    out["front_km"] = float(x[cold].max() / 1000.0) if cold.size else 0.0
    warm = np.where(tp[:, 0, :] > 0.1, tp[:, 0, :], 0.0)
    out["warm_centroid_km"] = float((z[:, None] * warm).sum() / max(warm.sum(), 1e-300) / 1000.0)
    rows = np.where((warm > 0).any(axis=1))[0]
    out["warm_top_km"] = float(z[rows.max()] / 1000.0) if rows.size else 0.0
    return out
