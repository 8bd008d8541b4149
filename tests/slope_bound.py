"""Pathwise FP64 bound for runs in which the density comes near zero.

The local noise amplitude is sqrt(c max(rho, 0)) (eq. xilocal, with the
zero-density clamp of Sec. IV).  Its slope 1/(2 sqrt(rho)) turns a rounding
difference in the pre-collision density rho into a noise difference; at
rho = rho_mean that slope is what the 1e-12 rho_mean bar allows for.  A run
whose density comes within |rho| of zero therefore gets the bar scaled by
sqrt(rho_mean / |rho|) at its closest approach, with |rho| floored at the
rounding of the Q-term FP64 density sum, Q 2^-53 sum_i |f_i|, below which the
two implementations may see opposite signs of rho.  The oracle is stepped one
step at a time to find that approach; the result equals one call of
oracle.run over all the steps."""
import numpy as np


def oracle_run_with_slope(orc, lat, dims, f0, nsteps, tau, rho_mean, seed, mode=None, dist=None, t0=0):
    """(f after nsteps, slope factor >= 1) for the oracle's run from f0."""
    mode = orc.NOISE_LOCAL if mode is None else mode
    dist = orc.GAUSSIAN if dist is None else dist
    f = np.array(f0, dtype=np.float64, copy=True)
    Q = f.shape[0]
    amp = 1.0
    for t in range(t0, t0 + nsteps):
        r = f.sum(0)
        floor = Q * 2.0 ** -53 * np.abs(f).sum(0)
        amp = max(amp, float(np.max(np.sqrt(rho_mean / np.maximum(np.abs(r), floor)))))
        f = orc.run(lat, dims, f, 1, tau, mode, dist, rho_eq=rho_mean, seed=seed, t0=t)
    return f, amp
