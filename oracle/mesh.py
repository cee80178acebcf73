"""Element geometry, metric terms and face connectivity for the oracle.

The paper runs on curved hexahedra (Section 3.1) without giving the geometry
treatment.  Readings taken here:

* Element map x(xi): tensor Lagrange interpolation of the (q+1)^dim nodes
  placed at equispaced reference points (q = 1 or 2).
* Metric terms S[d, i] = |J| d xi_d / d x_i at solution points and flux
  points are computed in conservative-curl form (Kopriva 2006): in 3D,
  S[d, n] = [curl_xi (x_l grad_xi x_m)]_d with (n, l, m) cyclic, where the
  product x_l grad_xi x_m is first interpolated on the (p+1)^3
  Gauss-Lobatto points and the curl is then taken exactly.  In 2D,
  S = [[y_eta, -x_eta], [-y_xi, x_xi]] from the same GLL interpolant.  The
  resulting S is a polynomial of degree <= p per direction, so the discrete
  divergence sum_d D_d S[d, :] vanishes (free-stream preservation) and the
  face-normal component depends only on data on that face (neighbours
  agree).
* |J| at solution points is det(dx/dxi) of the element map.
* One area-weighted normal per face point, taken from the side whose
  (element, face) pair is smaller; the other side uses its exact negative,
  so common fluxes are equal and opposite (discrete conservation).

Test infrastructure (see ``oracle/__init__``).
"""
from __future__ import annotations

import numpy as np

from .basis import Ref1D, lagrange, lagrange_deriv


def _apply(vals, mats, dim):
    """Apply 1D matrices along each direction of tensor data.

    vals: [..., n_{dim-1}, ..., n_0] (direction 0 is the last axis).
    mats[d]: [m_d, n_d] or None (identity).  Returns [..., m_{dim-1}, ..., m_0].
    """
    out = vals
    for d in range(dim):
        A = mats[d]
        if A is None:
            continue
        ax = out.ndim - 1 - d
        out = np.moveaxis(np.tensordot(out, A, axes=([ax], [1])), -1, ax)
    return out


def orientation_map(Np, dim, o):
    """Index into the neighbour's face points for each of this side's face points.

    dim=2: bit 0 reverses the order.  dim=3: face point (a, b) (a fastest);
    bit 2 swaps (a, b), then bit 0 reverses a and bit 1 reverses b.
    """
    if dim == 2:
        a = np.arange(Np)
        return (Np - 1 - a) if (o & 1) else a
    b, a = np.meshgrid(np.arange(Np), np.arange(Np), indexing="ij")
    a, b = a.ravel(), b.ravel()
    if o & 4:
        a, b = b, a
    if o & 1:
        a = Np - 1 - a
    if o & 2:
        b = Np - 1 - b
    return a + Np * b


class Mesh:
    """Geometry and connectivity of an FR mesh of uniform order p.

    Arrays (E elements, Nsp = Np^dim, Nfp = Np^(dim-1), nface = 2 dim):

    * ``xsp`` [E, Nsp, dim] physical solution-point coordinates
    * ``J`` [E, Nsp] Jacobian determinant at solution points
    * ``S`` [E, dim(d), dim(i), Nsp] metric terms |J| dxi_d/dx_i
    * ``N`` [E, nface, Nfp, dim] outward area-weighted normals at flux points
    * ``nbr`` [E, nface, 3] connectivity as given; ``fpmap[e, f]`` index of the
      neighbour face point matching each face point
    """

    def __init__(self, nodes, conn, p, kind=0):
        nodes = np.asarray(nodes, float)
        conn = np.asarray(conn, np.int64)
        E, nn, dim = nodes.shape
        q = int(round(nn ** (1.0 / dim))) - 1
        if (q + 1) ** dim != nn:
            raise ValueError("node count is not (q+1)^dim")
        self.dim, self.E, self.q, self.p = dim, E, q, p
        self.ref = Ref1D(p, kind)
        Np = p + 1
        self.Np, self.Nsp, self.Nfp, self.nface = Np, Np ** dim, Np ** (dim - 1), 2 * dim
        self.nodes, self.conn = nodes, conn
        ref = self.ref
        xe = np.linspace(-1.0, 1.0, q + 1)
        # nodal coordinates as tensors [E, dim(comp), (q+1)...]
        X = nodes.reshape((E,) + (q + 1,) * dim + (dim,))
        X = np.moveaxis(X, -1, 1)
        # Derivatives of the map and the conservative-curl products use
        # coordinates relative to the element's node centroid: both are
        # invariant under a translation (sum_a l_a' = 0, and the curl of
        # c grad x_m vanishes when the map lies in the interpolation space,
        # q <= p), and the relative coordinates avoid cancellation in
        # elements far from the origin.
        cen = nodes.mean(axis=1)                         # [E, dim]
        Xr = X - cen.reshape((E, dim) + (1,) * dim)

        def geo(pts, deriv=None, rel=False):
            mats = [lagrange(xe, pts[d]) if deriv != d else lagrange_deriv(xe, pts[d])
                    for d in range(dim)]
            return _apply(Xr if rel else X, mats, dim)

        gl = [ref.x] * dim
        self.xsp = np.moveaxis(geo(gl), 1, -1).reshape(E, -1, dim)
        A = np.stack([geo(gl, k, rel=True) for k in range(dim)], axis=2)  # [E, comp i, deriv k, ...]
        A = A.reshape(E, dim, dim, -1)
        self.J = np.linalg.det(np.moveaxis(A, -1, 1))  # [E, Nsp]
        if np.any(self.J <= 0.0):
            raise ValueError("non-positive Jacobian")
        # GLL values of the map and its derivatives (exact from the map)
        gll = [ref.gll] * dim
        xg = geo(gll, rel=True)                         # [E, i, gll...] (relative)
        ag = np.stack([geo(gll, k, rel=True) for k in range(dim)], axis=2)  # [E, i, k, gll...]

        def smetric(pts):
            """S[E, d, i, ...] evaluated on the tensor grid pts (list of 1D arrays)."""
            I = [lagrange(ref.gll, pts[d]) for d in range(dim)]
            Dm = [lagrange_deriv(ref.gll, pts[d]) for d in range(dim)]

            def ev(f, dk):
                mats = [Dm[d] if d == dk else I[d] for d in range(dim)]
                return _apply(f, mats, dim)

            shp = (E, dim, dim) + tuple(len(pts[d]) for d in reversed(range(dim)))
            S = np.zeros(shp)
            if dim == 2:
                x, y = xg[:, 0], xg[:, 1]
                S[:, 0, 0] = ev(y, 1)
                S[:, 0, 1] = -ev(x, 1)
                S[:, 1, 0] = -ev(y, 0)
                S[:, 1, 1] = ev(x, 0)
                return S
            for n in range(3):
                l, m = (n + 1) % 3, (n + 2) % 3
                w = [xg[:, l] * ag[:, m, k] for k in range(3)]  # x_l d x_m / d xi_k
                for d in range(3):
                    d1, d2 = (d + 1) % 3, (d + 2) % 3
                    S[:, d, n] = ev(w[d2], d1) - ev(w[d1], d2)
            return S

        self.S = smetric(gl).reshape(E, dim, dim, -1)
        # normals at flux points of each face, from this element's own metric
        Nown = np.zeros((E, self.nface, self.Nfp, dim))
        for d in range(dim):
            for side in (0, 1):
                pts = [ref.x] * dim
                pts[d] = np.array([1.0 if side else -1.0])
                Sf = smetric(pts)[:, d]           # [E, i, ...]
                Sf = Sf.reshape(E, dim, -1)
                sgn = 1.0 if side else -1.0
                Nown[:, 2 * d + side] = sgn * np.moveaxis(Sf, 1, 2)
        self.Nown = Nown
        # connectivity: neighbour face-point maps and shared normals
        self.fpmap = np.zeros((E, self.nface, self.Nfp), np.int64)
        N = Nown.copy()
        for e in range(E):
            for f in range(self.nface):
                ne, nf, o = conn[e, f]
                if ne < 0:
                    self.fpmap[e, f] = np.arange(self.Nfp)
                    continue
                mp = orientation_map(Np, dim, int(o))
                self.fpmap[e, f] = mp
                back = conn[ne, nf]
                if back[0] != e or back[1] != f:
                    raise ValueError("connectivity is not symmetric")
                if (e, f) > (int(ne), int(nf)):
                    N[e, f] = -Nown[ne, nf][mp]
        self.N = N
        self.normal_mismatch = float(np.max(np.abs(N - Nown))) if E else 0.0

    # ---- helpers used by the residual ---------------------------------
    def sp_tensor(self, a):
        """[..., Nsp] -> [..., Np, (Np,) Np] with direction 0 last."""
        return a.reshape(a.shape[:-1] + (self.Np,) * self.dim)

    def face_weights(self):
        """GL tensor quadrature weights of the face points [Nfp]."""
        w = self.ref.w
        if self.dim == 2:
            return w.copy()
        return np.outer(w, w).ravel()  # b slow, a fast

    def sp_weights(self):
        w = self.ref.w
        if self.dim == 2:
            return np.outer(w, w).ravel()
        return np.einsum("k,j,i->kji", w, w, w).ravel()

    def bc_faces(self, tag):
        """(element, face) index arrays of the boundary faces with the given tag."""
        m = self.conn[:, :, 0] == -tag
        e, f = np.nonzero(m)
        return e, f
