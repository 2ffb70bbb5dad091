"""Isoparametric geometry and face matching of a mesh given by its node coordinates (oracle; test
infrastructure only).

Sec. 3.1 uses k-th degree curved elements: the map of every element is the degree-k polynomial
interpolant of its GLL node positions X[e, d, i] (node i = a + n b + n^2 c, a along xi_1). The
node positions themselves are an input (the workload's mesh, from paper_2306_01085_gb300.workloads);
everything derived from them here (Jacobians, normals, neighbours) is computed independently of the
library.

Jacobians are taken of X - X[:, :, 0] (the element's first node): the derivatives of the basis sum
to zero, so this is the same quantity, but its rounding is relative to the element size rather than
to |x| (a 2.5 km layer at 6471 km radius would otherwise lose four digits).

Face matching is done here by brute force on physical coordinates (face centres, then nearest face
quadrature point), independently of the library's bookkeeping.

Pinned by tests/test_oracle_mesh.py: element volumes / shell volume, closed-surface normal sums,
outward orientation, matched points coincide, first-layer height and layer sum.
"""
import math

import numpy as np
from scipy.spatial import cKDTree

from paper_2306_01085_gb300 import workloads as W

from . import quadrature as Q

BC_INTERIOR, BC_WALL, BC_OUTFLOW = 0, 1, 2


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
        self.X = W.mesh_nodes(desc) if X is None else X
        self.n_elem = self.X.shape[0]
        self._geometry()
        self._connect()

    # -- geometry ---------------------------------------------------------------------------
    def _geometry(self):
        X = self.X
        Xr = X - X[:, :, :1]                                           # relative to the first node
        # J[e, g, d, a] = d x_d / d xi_a at volume Gauss points
        J = np.einsum("edi,gai->egda", Xr, self.dphi)
        self.detJ = np.linalg.det(J)
        self.Jinv = np.linalg.inv(J)                                   # [e, g, a, d] = d xi_a / d x_d
        self.xG = np.einsum("edi,gi->edg", X, self.phi)
        nF, xF = [], []
        for f, (axis, side) in enumerate(Q.FACES):
            Jf = np.einsum("edi,gai->egda", Xr, self.dphiF[f])
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
