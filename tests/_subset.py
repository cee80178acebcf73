"""Oracle residual of a sample of elements of a large mesh.

The residual of element s depends only on its own state and, through each
shared face, on the neighbour's trace and the neighbour's BR2 face flux at
that face (itself a function of the neighbour's state and that face's jump).
So R restricted to the sample equals the residual of the sample computed on
the sub-mesh of the sample plus its face neighbours, with every face that
leaves the sub-mesh closed by a wall (which only changes the neighbours' own
residuals, which are discarded).
"""
import numpy as np

from paper_2501_05709_gb300 import workloads as W


def submesh(nodes, conn, sample):
    sample = np.unique(np.asarray(sample, np.int64))
    keep = set(sample.tolist())
    for e in sample:
        for f in range(conn.shape[1]):
            if conn[e, f, 0] >= 0:
                keep.add(int(conn[e, f, 0]))
    ids = np.array(sorted(keep), np.int64)
    loc = {int(e): i for i, e in enumerate(ids)}
    sub_conn = conn[ids].copy()
    for i in range(len(ids)):
        for f in range(conn.shape[1]):
            nb = int(sub_conn[i, f, 0])
            if nb >= 0:
                if nb in loc:
                    sub_conn[i, f, 0] = loc[nb]
                else:
                    sub_conn[i, f] = (-W.BC_WALL, 0, 0)
    pos = np.array([loc[int(e)] for e in sample], np.int64)
    return nodes[ids], sub_conn, ids, pos


def sampled_residual(make_solver, nodes, conn, u_full_fn, sample):
    """R of the sampled elements.  make_solver(nodes, conn) -> (mesh, solver);
    u_full_fn(ids, mesh) -> state of the sub-mesh elements [n, nvar, Nsp]."""
    sub_nodes, sub_conn, ids, pos = submesh(nodes, conn, sample)
    m, s = make_solver(sub_nodes, sub_conn)
    u = u_full_fn(ids, m)
    return s.residual(u)[pos], np.unique(np.asarray(sample, np.int64))
