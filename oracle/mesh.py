"""Meshes, isoparametric geometry and face matching (oracle; test infrastructure only).

Sec. 3.1 uses k-th degree curved elements; Sec. 3.3 uses cubed-sphere shells with geometric radial
growth from a first-layer height. The map of every element is the degree-k polynomial interpolant
of its GLL node positions (isoparametric). Conventions shared with the library (stated in
include/dg.h, implemented separately on each side):

  box   element e = i + nx (j + ny k); nodes at x = (i + (1 + xi_a)/2) lx/nx, ...
  shell element e = k + nz (i + n (j + n P)) for panel P, angular cell (i, j), radial layer k;
        equiangular gnomonic panels: direction c_P + tan(alpha) a_P + tan(beta) b_P, normalised,
        alpha, beta in [-pi/4, pi/4]; panels (c, a, b) =
        (+x,+y,+z) (+y,-x,+z) (-x,-y,+z) (-y,+x,+z) (+z,+y,-x) (-z,+y,+x).
  node  i = a + n b + n^2 c (a along xi_1, the fastest), n = k+1.

Face matching is done here by brute force on physical coordinates (face centres, then nearest face
quadrature point), independently of the library's bookkeeping.

Pinned by tests/test_oracle_mesh.py: element volumes / shell volume, closed-surface normal sums,
outward orientation, matched points coincide, first-layer height and layer sum.
"""
import math

import numpy as np
from scipy.spatial import cKDTree

from . import quadrature as Q

PANELS = [
    ((1, 0, 0), (0, 1, 0), (0, 0, 1)),
    ((0, 1, 0), (-1, 0, 0), (0, 0, 1)),
    ((-1, 0, 0), (0, -1, 0), (0, 0, 1)),
    ((0, -1, 0), (1, 0, 0), (0, 0, 1)),
    ((0, 0, 1), (0, 1, 0), (-1, 0, 0)),
    ((0, 0, -1), (0, 1, 0), (1, 0, 0)),
]

BC_INTERIOR, BC_WALL, BC_OUTFLOW = 0, 1, 2


def radial_layers(r_in, r_out, nz, h_first):
    """Layer interfaces r_0 = r_in < ... < r_nz = r_out with heights h_first q^k (Sec. 3.3).

    The growth ratio q solves sum_{k<nz} h_first q^k = r_out - r_in (bisection); h_first <= 0 gives
    uniform layers.
    """
    total = r_out - r_in
    if h_first <= 0.0 or nz == 1:
        return r_in + total * np.arange(nz + 1) / nz
    def excess(q):
        return h_first * sum(q ** k for k in range(nz)) - total
    lo, hi = 1.0, 2.0
    if excess(lo) > 0:
        lo, hi = 1e-6, 1.0
    while excess(hi) < 0:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if excess(mid) > 0:
            hi = mid
        else:
            lo = mid
    q = 0.5 * (lo + hi)
    r = r_in + np.concatenate([[0.0], np.cumsum(h_first * q ** np.arange(nz))])
    r[-1] = r_out
    return r


def node_coordinates(desc):
    """GLL node positions X[e, d, i] of every element (isoparametric node set)."""
    n = desc.p + 1
    xi, _ = Q.gll(n)
    ref = Q.tensor_points(xi)          # (n^3, 3): (xi_a, xi_b, xi_c)
    s = 0.5 * (1.0 + ref)              # in [0, 1]
    if desc.kind == 0:
        hx, hy, hz = desc.lx / desc.nx, desc.ly / desc.ny, desc.lz / desc.nz
        X = np.zeros((desc.n_elem, 3, n ** 3))
        for k in range(desc.nz):
            for j in range(desc.ny):
                for i in range(desc.nx):
                    e = i + desc.nx * (j + desc.ny * k)
                    X[e, 0] = (i + s[:, 0]) * hx
                    X[e, 1] = (j + s[:, 1]) * hy
                    X[e, 2] = (k + s[:, 2]) * hz
        return X
    nn, nz = desc.nx, desc.nz
    rl = radial_layers(desc.r_inner, desc.r_outer, nz, desc.h_first)
    d_ang = 0.5 * math.pi / nn
    X = np.zeros((desc.n_elem, 3, n ** 3))
    for P, (c, a, b) in enumerate(PANELS):
        c, a, b = np.array(c, float), np.array(a, float), np.array(b, float)
        for j in range(nn):
            for i in range(nn):
                alpha = -0.25 * math.pi + (i + s[:, 0]) * d_ang
                beta = -0.25 * math.pi + (j + s[:, 1]) * d_ang
                dirv = c[:, None] + np.tan(alpha)[None, :] * a[:, None] + np.tan(beta)[None, :] * b[:, None]
                dirv = dirv / np.sqrt((dirv ** 2).sum(0))[None, :]
                for k in range(nz):
                    e = k + nz * (i + nn * (j + nn * P))
                    r = rl[k] + s[:, 2] * (rl[k + 1] - rl[k])
                    X[e] = dirv * r[None, :]
    return X


class OracleMesh:
    """Reference operators, geometry at quadrature points and face neighbours of one mesh."""

    def __init__(self, desc, X=None):
        self.desc = desc
        self.p = desc.p
        self.n = n = desc.p + 1
        self.Np = n ** 3
        self.Nf = n * n
        self.xi, _ = Q.gll(n)
        self.xg, self.wg = Q.gauss(n)
        gpts = Q.tensor_points(self.xg)
        self.phi, self.dphi = Q.basis3d(self.xi, gpts)               # (g, i), (g, 3, i)
        self.W = np.einsum("c,b,a->cba", self.wg, self.wg, self.wg).ravel()
        self.phiF, self.dphiF = [], []
        for f in range(6):
            ph, dph = Q.basis3d(self.xi, Q.face_points(self.xg, f))
            self.phiF.append(ph)
            self.dphiF.append(dph)
        self.wF = np.einsum("b,a->ba", self.wg, self.wg).ravel()
        self.X = node_coordinates(desc) if X is None else X
        self.n_elem = self.X.shape[0]
        self._geometry()
        self._connect()

    # -- geometry ---------------------------------------------------------------------------
    def _geometry(self):
        X = self.X
        # J[e, g, d, a] = d x_d / d xi_a at volume Gauss points
        J = np.einsum("edi,gai->egda", X, self.dphi)
        self.detJ = np.linalg.det(J)
        self.Jinv = np.linalg.inv(J)                                   # [e, g, a, d] = d xi_a / d x_d
        self.xG = np.einsum("edi,gi->edg", X, self.phi)
        nF, xF = [], []
        for f, (axis, side) in enumerate(Q.FACES):
            Jf = np.einsum("edi,gai->egda", X, self.dphiF[f])
            t1 = Jf[..., (axis + 1) % 3]
            t2 = Jf[..., (axis + 2) % 3]
            nF.append(side * np.moveaxis(np.cross(t1, t2), -1, 1))    # (e, 3, f) outward n dS
            xF.append(np.einsum("edi,fi->edf", X, self.phiF[f]))
        self.nF = np.stack(nF, axis=1)                                 # (e, 6, 3, Nf)
        self.xF = np.stack(xF, axis=1)
        self.areaF = np.sqrt((self.nF ** 2).sum(2))                    # (e, 6, Nf)

    def _periods(self):
        d = self.desc
        if d.kind != 0:
            return [0.0, 0.0, 0.0]
        return [d.lx, d.ly, d.lz if d.bc_lo == 0 else 0.0]

    def _wrap(self, diff):
        for a, L in enumerate(self._periods()):
            if L > 0:
                diff[..., a, :] = diff[..., a, :] - L * np.round(diff[..., a, :] / L)
        return diff

    def _connect(self):
        d = self.desc
        n, E = self.n, self.n_elem
        # corner nodes of each local face (GLL includes the end points)
        idx = np.arange(self.Np).reshape(n, n, n)                      # [c, b, a]
        corner_sets = []
        for axis, side in Q.FACES:
            k = 0 if side < 0 else n - 1
            sl = [slice(None)] * 3
            sl[2 - axis] = k
            face_nodes = idx[tuple(sl)]
            corner_sets.append([face_nodes[0, 0], face_nodes[0, -1], face_nodes[-1, 0], face_nodes[-1, -1]])
        centres = np.stack([self.X[:, :, cs].mean(-1) for cs in corner_sets], axis=1)   # (E, 6, 3)
        per = self._periods()
        scale = float(np.abs(self.X).max()) + 1.0
        tol = 1e-7 * scale
        pts = centres.reshape(-1, 3).copy()
        box = np.zeros(3)
        for a in range(3):
            if per[a] > 0:
                pts[:, a] = np.mod(pts[:, a], per[a])
                pts[:, a] = np.where(per[a] - pts[:, a] < tol, 0.0, pts[:, a])
                box[a] = per[a]
            else:
                shift = pts[:, a].min() - 1.0
                pts[:, a] -= shift
                box[a] = 4.0 * (pts[:, a].max() + 1.0)
        tree = cKDTree(pts, boxsize=box)
        dist, nn = tree.query(pts, k=2)
        self.nbr_elem = np.full((E, 6), -1, dtype=np.int64)
        self.nbr_face = np.full((E, 6), -1, dtype=np.int64)
        table = {}
        for idx_flat in range(E * 6):
            e, f = divmod(idx_flat, 6)
            other = nn[idx_flat, 1] if nn[idx_flat, 0] == idx_flat else nn[idx_flat, 0]
            dd = dist[idx_flat, 1] if nn[idx_flat, 0] == idx_flat else dist[idx_flat, 0]
            if dd < tol:
                self.nbr_elem[e, f], self.nbr_face[e, f] = divmod(int(other), 6)
            else:
                table[(e, f)] = (e, f)
        # boundary kinds of the faces left unmatched
        self.bc = np.zeros((E, 6), dtype=np.int64)
        for (e, f) in table.values():
            cs = corner_sets[f]
            if d.kind == 0:
                z = self.X[e, 2, cs].mean()
                self.bc[e, f] = d.bc_lo if abs(z) < tol else d.bc_hi
            else:
                r = np.sqrt((self.X[e][:, cs] ** 2).sum(0)).mean()
                self.bc[e, f] = d.bc_lo if abs(r - d.r_inner) < abs(r - d.r_outer) else d.bc_hi
        if np.any((self.nbr_elem < 0) & (self.bc == 0)):
            raise RuntimeError("unmatched face without a boundary condition")
        # point matching: nearest neighbour face quadrature point (with periodic wrap)
        self.nbr_pt = np.zeros((E, 6, self.Nf), dtype=np.int64)
        for f in range(6):
            inter = np.nonzero(self.nbr_elem[:, f] >= 0)[0]
            for chunk in np.array_split(inter, max(1, len(inter) // 2048)):
                if len(chunk) == 0:
                    continue
                e2 = self.nbr_elem[chunk, f]
                f2 = self.nbr_face[chunk, f]
                own = self.xF[chunk, f]                                # (m, 3, Nf)
                oth = self.xF[e2, f2]                                  # (m, 3, Nf)
                diff = own[:, :, :, None] - oth[:, :, None, :]         # (m, 3, Nf, Nf)
                diff = self._wrap(diff.reshape(len(chunk), 3, -1)).reshape(diff.shape)
                dist = (diff ** 2).sum(1)
                self.nbr_pt[chunk, f] = np.argmin(dist, axis=-1)
                self.match_err = max(getattr(self, "match_err", 0.0), float(np.sqrt(dist.min(-1).max())))

    def neighbours(self, elems):
        """Face neighbours of a set of elements (interior faces only)."""
        nb = self.nbr_elem[np.asarray(elems)]
        return np.unique(nb[nb >= 0])
