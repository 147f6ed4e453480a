"""Measurements of a (2+1)D state split by a Klein step at x0 (for the
refraction tests): probability, centroid and mean local wave vector of the
transmitted (x > x0) and reflected parts.  Not used by the oracle or the
library."""
import numpy as np

from paper_1309_3452_gb300 import workloads as W


def parts(prob, psi, x0):
    """{'T': (weight, centroid (x, y), mean k (kx, ky)), 'R': ...}; k from the
    phase gradient Im(conj(psi) d psi) of each plane along its own cell grid,
    summed over the planes (every component of a plane wave carries the same
    exp(i k.x))."""
    acc = {key: np.zeros(5) for key in "TR"}
    for pl in range(prob.n_planes):
        xyz = W.site_positions(prob, pl)
        v = psi[pl, 0]
        x = np.broadcast_to(xyz[0], psi[pl].shape)[0]
        y = np.broadcast_to(xyz[1], psi[pl].shape)[0]
        d = np.abs(v) ** 2
        # centred differences across one cell: Im(conj(v) dv) / dx
        gx = np.imag(np.conj(v) * (np.roll(v, -1, axis=1) - np.roll(v, 1, axis=1))) / (2 * prob.dx[0])
        gy = np.imag(np.conj(v) * (np.roll(v, -1, axis=0) - np.roll(v, 1, axis=0))) / (2 * prob.dx[1])
        for key, m in (("T", x > x0), ("R", x <= x0)):
            acc[key] += [d[m].sum(), (d * x)[m].sum(), (d * y)[m].sum(), gx[m].sum(), gy[m].sum()]
    out = {}
    for key, a in acc.items():
        w = max(a[0], 1e-300)
        out[key] = (a[0], np.array([a[1] / w, a[2] / w]), np.array([a[3] / w, a[4] / w]))
    return out


def velocity(prob, p1, p2, nsteps, x0):
    """Centroid velocity of each part between two states nsteps apart."""
    a, b = parts(prob, p1, x0), parts(prob, p2, x0)
    return {key: (b[key][1] - a[key][1]) / (nsteps * prob.dt) for key in "TR"}, b
