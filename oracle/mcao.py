"""MCAO fitting of the reconstructed layers onto several deformable mirrors
(Sec. 5: the 9-layer MCAO case solves the fitting equation with an
unpreconditioned CG of 4 iterations; the mirrors of the paper's MCAO system
are 85x85 at 0 m with 0.5 m pitch, 47x47 at 4 km and 53x53 at 12.7 km with
1 m pitch, table of system settings).

TEST INFRASTRUCTURE ONLY: plain FP64 numpy, dense one-dimensional interpolation
matrices, written for checking, never for speed.

Reading (the paper names the fitting step but not its operator): the mirror
shapes a = (a_1 .. a_D) minimise sum_t || P^DM_t a - P^L_t phi ||^2 over the
fitting directions theta_t, where phi = W^{-1} c are the reconstructed layers,
P^L_t projects every layer onto the pupil nodes in direction theta_t (no cone)
and sums them, and P^DM_t does the same for the mirrors; both are bilinear on
their grids.  Mirror d has n_d x n_d actuators with pitch s_d centred on the
axis (actuator i at x = (i - (n_d - 1)/2) s_d) at altitude h_d.  The normal
equations N a = b, N = sum_t P^DM_t^T P^DM_t, b = sum_t P^DM_t^T P^L_t phi,
are solved by `iters` iterations of CG without preconditioner from the
caller's start a_0.
"""
import numpy as np

from .oracle import dwt2_inv


def interp_matrix(xs, spacing, centre, n):
    """Rows: points xs; columns: grid nodes 0..n-1 at (k - centre) * spacing.
    Bilinear (hat) weights; a point outside [0, n-1] grid units is an error."""
    f = np.asarray(xs, dtype=np.float64) / spacing + centre
    k = np.floor(f).astype(int)
    if np.any(k < 0) or np.any(k + 1 > n - 1):
        raise ValueError("projection outside the grid")
    w = f - k
    M = np.zeros((len(f), n))
    M[np.arange(len(f)), k] += 1.0 - w
    M[np.arange(len(f)), k + 1] += w
    return M


class McaoFit:
    """dms: list of (n_act, pitch, altitude); dirs: list of (theta_x, theta_y)."""

    def __init__(self, oracle, geom, dms, dirs):
        self.o, self.geom = oracle, geom
        self.dms, self.dirs = list(dms), list(dirs)
        self.m = geom.n_sub + 1
        ds = geom.D / geom.n_sub
        x = -0.5 * geom.D + ds * np.arange(self.m)  # pupil node coordinates
        # layer grids: node k at (k - n/2) d_l (the oracle's layer spacing)
        self.lay = []
        for l, ly in enumerate(geom.layers):
            d = oracle.layer_spacing(l)
            self.lay.append([(interp_matrix(x + ly.h * ty, d, 0.5 * ly.n, ly.n),
                              interp_matrix(x + ly.h * tx, d, 0.5 * ly.n, ly.n)) for tx, ty in self.dirs])
        self.dm = []
        for n_act, pitch, h in self.dms:
            c = 0.5 * (n_act - 1)
            self.dm.append([(interp_matrix(x + h * ty, pitch, c, n_act),
                             interp_matrix(x + h * tx, pitch, c, n_act)) for tx, ty in self.dirs])
        self.sizes = [n * n for n, _, _ in self.dms]

    @property
    def n_actuators(self):
        return sum(self.sizes)

    def split(self, a):
        out, o = [], 0
        for (n, _, _), sz in zip(self.dms, self.sizes):
            out.append(np.asarray(a[o:o + sz], dtype=np.float64).reshape(n, n))
            o += sz
        return out

    def nodal(self, c):
        """phi = W^{-1} c, layer by layer (row index = y)."""
        taps = self.o.taps
        out, o = [], 0
        for ly in self.geom.layers:
            sz = ly.n * ly.n
            out.append(dwt2_inv(np.asarray(c[o:o + sz]).reshape(ly.n, ly.n), ly.J, taps) / ly.delta)
            o += sz
        return out

    def project_layers(self, layers):
        """P^L_t phi for every direction: array [T][m][m]."""
        return np.array([sum(My @ L @ Mx.T for L, (My, Mx) in zip(layers, [tabs[t] for tabs in self.lay]))
                         for t in range(len(self.dirs))])

    def project_dms(self, a):
        """P^DM_t a for every direction: array [T][m][m]."""
        A = self.split(a)
        return np.array([sum(My @ Ad @ Mx.T for Ad, (My, Mx) in zip(A, [tabs[t] for tabs in self.dm]))
                         for t in range(len(self.dirs))])

    def project_dms_T(self, y):
        """sum_t P^DM_t^T y_t, as one actuator vector."""
        parts = []
        for tabs in self.dm:
            parts.append(sum(My.T @ y[t] @ Mx for t, (My, Mx) in enumerate(tabs)).ravel())
        return np.concatenate(parts)

    def normal(self, a):
        return self.project_dms_T(self.project_dms(a))

    def rhs(self, c):
        return self.project_dms_T(self.project_layers(self.nodal(c)))

    def fit(self, c, a0, iters):
        """`iters` CG iterations on N a = b from a0 (no preconditioner)."""
        b = self.rhs(c)
        a = np.array(a0, dtype=np.float64)
        r = b - self.normal(a)
        p = r.copy()
        rr = r @ r
        for _ in range(iters):
            if rr == 0.0:
                break
            q = self.normal(p)
            alpha = rr / (p @ q)
            a += alpha * p
            r -= alpha * q
            rr_new = r @ r
            p = r + (rr_new / rr) * p
            rr = rr_new
        return a

    def residual(self, c, a):
        """sum_t || P^DM_t a - P^L_t phi ||^2"""
        e = self.project_dms(a) - self.project_layers(self.nodal(c))
        return float(np.sum(e * e))


def paper_mirrors():
    """The paper's MCAO mirrors: (actuators per side, pitch [m], altitude [m])."""
    return [(85, 0.5, 0.0), (47, 1.0, 4000.0), (53, 1.0, 12700.0)]


def fitting_directions(radius_arcmin=0.25, k=6):
    """Reading: the optical axis and k directions on a circle of the given
    radius.  The paper does not list its fitting directions; 0.25 arcmin keeps
    every projection inside the reconstructed layer grids of the ELT workload
    (their extent is set by the guide stars' cones)."""
    r = radius_arcmin * np.pi / (180.0 * 60.0)
    return [(0.0, 0.0)] + [(r * np.cos(2 * np.pi * i / k), r * np.sin(2 * np.pi * i / k)) for i in range(k)]
