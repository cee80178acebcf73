"""Pins of the degree-q elements inside a degree-p mesh (oracle.mixed, the
variable solution degree of Section 3.1): the mortar operators against their
closed forms, the degree-q path at q = p against the uniform scheme, linear
advection on a uniformly reduced mesh against the uniform degree-q scheme,
exact BR2 face gradients of a degree-q state, conservation on a curved mesh
and a free stream on an affine one."""
import math

import numpy as np
import pytest

from oracle import mixed as MX
from oracle import sponge as SP
from oracle.basis import DG, HUYNH_G2, gauss_legendre
from oracle.fr import FRSolver
from oracle.mesh import Mesh
from oracle.physics import Advection, NavierStokes
from paper_2501_05709_gb300 import workloads as W


def _box(p, n=3, curve=0.0, q=1, seed=2, kind=DG, dim=3):
    nodes, conn = W.box_mesh(dim, n, 0.0, 2 * math.pi, q=q, curve=curve, seed=seed)
    return Mesh(nodes, conn, p, kind=kind)


def _state(m, seed):
    return np.ascontiguousarray(np.moveaxis(W.random_smooth_state(m.xsp, seed=seed), 0, 1))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mortar_operators(p):
    xp, wp = gauss_legendre(p + 1)
    for q in range(p + 1):
        ops = MX.MortarOps(p, q, DG)
        xq, wq = gauss_legendre(q + 1)
        assert np.allclose(ops.Iqp @ ops.Ipq, np.eye(q + 1), atol=1e-13)     # q -> p -> q is the identity
        for k in range(q + 1):
            assert np.allclose(ops.Iqp @ xp ** k, xq ** k, atol=1e-13)        # interpolation exact to degree q
            assert np.allclose(ops.Ipq @ xq ** k, xp ** k, atol=1e-13)
            assert np.allclose(ops.Pqp @ xp ** k, xq ** k, atol=1e-13)        # projection exact to degree q
        for k in range(q + 1, p + 1):                                          # and blind to P_{q+1..p}
            assert np.allclose(ops.Pqp @ SP.legendre_values(k, xp), 0.0, atol=1e-13)
        f = np.cos(3.0 * xp) + xp ** p
        assert abs(wq @ (ops.Pqp @ f) - wp @ f) <= 1e-13                      # the face mean is kept
        if q == 0:   # the one linear correction function, whatever the kind
            for kind in (DG, HUYNH_G2):
                r0 = MX.MortarOps(p, 0, kind).ref
                assert np.allclose(r0.hm, [0.5]) and np.allclose(r0.hp, [0.5]) and np.allclose(r0.D, [[0.0]])


@pytest.mark.parametrize("kind", [DG, HUYNH_G2])
def test_degree_p_path_is_the_uniform_scheme(kind):
    # the reduced-element formulas with q = p on every element of a curved,
    # viscous mesh give the uniform scheme's face gradients and residual
    m = _box(3, curve=0.1, q=2, kind=kind)
    ph = NavierStokes(3, mu=0.02)
    u = _state(m, 7)
    s = FRSolver(m, ph)
    R, faces = s.residual(u, want_faces=True)
    ops = MX.MortarOps(3, 3, kind)
    sel = np.arange(m.E)
    # rebuild the face inputs of the uniform scheme
    uf = faces["uf"]
    jmp = np.zeros_like(uf)
    ei, fi = np.nonzero(m.conn[:, :, 0] >= 0)
    ne, nfc = m.conn[ei, fi, 0], m.conn[ei, fi, 1]
    uo = np.moveaxis(uf[ne[:, None], nfc[:, None], :, m.fpmap[ei, fi]], -1, 1)
    jmp[ei, fi] = 0.5 * (uo - uf[ei, fi])
    G = MX.face_gradients(m, ph, sel, ops, u, jmp)
    assert np.abs(G - faces["Gface"]).max() <= 1e-11 * np.abs(faces["Gface"]).max()
    uR = np.zeros_like(uf)
    uR[ei, fi] = uo                                     # periodic: every face has a neighbour
    Fc = np.moveaxis(ph.rusanov(np.moveaxis(uf, 2, 0), np.moveaxis(uR, 2, 0), np.moveaxis(m.N, 3, 0)), 0, 2) \
        - faces["Fv_common"]
    Rr, Rq, Jq = MX.residual(m, ph, sel, ops, u, jmp, Fc)
    assert np.abs(Rr - R).max() <= 1e-11 * np.abs(R).max()
    assert np.allclose(Rq, R, rtol=0, atol=1e-11 * np.abs(R).max()) and np.allclose(Jq, m.J)


@pytest.mark.parametrize("p,q", [(2, 1), (3, 2), (3, 0), (4, 2)])
def test_linear_advection_equals_the_uniform_degree_q_scheme(p, q):
    # upwind fluxes of degree-q traces are degree-q face polynomials, so on an
    # affine mesh a mesh of degree-q elements with degree-p faces is the
    # uniform degree-q scheme
    a = np.array([0.6, -0.3, 0.45])
    mp, mq = _box(p, n=3), _box(q, n=3)
    rng = np.random.default_rng(p * 10 + q)
    uq = rng.standard_normal((mq.E, 1, mq.Nsp))
    ops = MX.MortarOps(p, q, DG)
    up = MX.volume(uq, ops.Ipq, 3)                      # the same polynomials at the degree-p points
    Rp = FRSolver(mp, Advection(a), caps=np.full(mp.E, q)).residual(up)
    Rq = FRSolver(mq, Advection(a)).residual(uq)
    assert np.abs(MX.volume(Rp, ops.Iqp, 3) - Rq).max() <= 1e-12 * np.abs(Rq).max()
    assert np.abs(MX.volume(Rq, ops.Ipq, 3) - Rp).max() <= 1e-12 * np.abs(Rq).max()


def test_face_gradients_of_a_degree_q_state_are_exact():
    # a conserved state linear in x on an affine box (p = 3, degrees 1..3):
    # on faces where it is continuous the BR2 face gradient is its gradient
    m = _box(3, n=3)
    ph = NavierStokes(3, mu=0.02)
    caps = np.random.default_rng(4).integers(1, 4, m.E)
    A = np.array([[1.2, 0.05, -0.03, 0.02], [0.3, 0.02, 0.04, -0.01], [-0.1, 0.01, 0.03, 0.05],
                  [0.2, -0.02, 0.01, 0.04], [3.0, 0.1, -0.05, 0.08]])     # u_v = A[v,0] + A[v,1:].x
    x = m.xsp
    u = np.einsum("vi,esi->evs", A[:, 1:], x) + A[:, 0][None, :, None]
    _, faces = FRSolver(m, ph, caps=caps).residual(u, want_faces=True)
    G = faces["Gface"]
    # a face is continuous unless it lies on the periodic seam (coordinate jump)
    xf = np.zeros((m.E, m.nface, m.Nfp, 3))
    for d in range(3):
        for s in (0, 1):
            lv = m.ref.lp if s else m.ref.lm
            t = x.reshape((m.E,) + (4, 4, 4) + (3,))
            xf[:, 2 * d + s] = np.tensordot(t, lv, axes=([3 - d], [0])).reshape(m.E, -1, 3)
    checked = 0
    for e in range(m.E):
        for f in range(m.nface):
            ne, nf, _ = m.conn[e, f]
            xo = xf[ne, nf][m.fpmap[e, f]]
            if np.abs(xo - xf[e, f]).max() > 1e-9:
                continue
            assert np.abs(G[e, f] - A[:, 1:, None]).max() <= 1e-12, (e, f, caps[e])
            checked += caps[e] < 3
    assert checked >= 20


def test_conservation_on_a_curved_mesh():
    # sum over elements of the integral of |J| R (degree-q quadrature on the
    # reduced elements) vanishes on a periodic curved mesh
    m = _box(3, curve=0.1, q=2)
    ph = NavierStokes(3, mu=0.02)
    caps = np.random.default_rng(2).integers(0, 4, m.E)
    u = SP.project(m, _state(m, 9), caps)
    s = FRSolver(m, ph, caps=caps)
    R, faces = s.residual(u, want_faces=True)
    full = caps == 3
    tot = np.einsum("evs,es,s->v", R[full], m.J[full], m.sp_weights())
    scale = np.einsum("evs,es,s->v", np.abs(R[full]), m.J[full], m.sp_weights()).max()
    for sel, q, Rq, Jq in faces["reduced"]:
        xq, wq = gauss_legendre(q + 1)
        w3 = np.einsum("k,j,i->kji", wq, wq, wq).ravel()
        tot = tot + np.einsum("evs,es,s->v", Rq, Jq, w3)
        scale = max(scale, np.einsum("evs,es,s->v", np.abs(Rq), Jq, w3).max())
    assert np.all(np.abs(tot) <= 1e-13 * scale)


def test_free_stream_on_an_affine_mixed_mesh():
    # turned element frames (all face orientation codes) on an affine box
    nodes, conn = W.box_mesh(3, 3, 0.0, 2 * math.pi, q=1)
    tn, tc, _ = W.reorient(nodes, conn, 3, seed=4)
    m = Mesh(tn, tc, 3)
    ph = NavierStokes(3, mu=0.01)
    caps = np.random.default_rng(0).integers(0, 4, m.E)
    u = W.perturbed_uniform(m.E, m.Nsp, 1.1, [0.3, -0.2, 0.1], 2.0, amplitude=0.0)
    R = FRSolver(m, ph, caps=caps).residual(u)
    assert np.max(np.abs(R)) < 1e-12


def test_source_needs_full_degree_elements():
    m = _box(2, n=2)
    with pytest.raises(ValueError):
        FRSolver(m, NavierStokes(3, mu=0.0), source=[(1.0, 1.0, (0, 0, 0), 1.0)], caps=np.zeros(m.E, int))


def _jumps(m, u):
    """Traces u_f and jumps u_c - u_f [E, nface, nv, Nfp] on a periodic mesh."""
    s = FRSolver(m, NavierStokes(m.dim, mu=0.01))
    _, faces = s.residual(u, want_faces=True)
    uf = faces["uf"]
    ei, fi = np.nonzero(m.conn[:, :, 0] >= 0)
    ne, nfc = m.conn[ei, fi, 0], m.conn[ei, fi, 1]
    uo = np.zeros_like(uf)
    uo[ei, fi] = np.moveaxis(uf[ne[:, None], nfc[:, None], :, m.fpmap[ei, fi]], -1, 1)
    return uf, 0.5 * (uo - uf)


def test_corrected_gradient_integrates_to_the_common_solution():
    # on an affine element of degree q the degree-q quadrature of |J| grad u
    # equals the face integral of u_c N at the degree-p face points: the
    # projected jumps keep each face's mean
    m = _box(3, n=3)
    caps = np.random.default_rng(6).integers(0, 3, m.E)
    u = SP.project(m, _state(m, 12), caps)
    uf, jmp = _jumps(m, u)
    uc = uf + jmp
    wf = m.face_weights()
    for q in range(3):
        sel = np.nonzero(caps == q)[0]
        ops = MX.MortarOps(3, q, DG)
        grad = MX.gradient(m, sel, ops, u, jmp)
        _, Jq = MX.metrics(m, sel, ops)
        xq, wq = gauss_legendre(q + 1)
        w3 = np.einsum("k,j,i->kji", wq, wq, wq).ravel()
        lhs = np.einsum("kvin,kn,n->kvi", grad, Jq, w3)
        rhs = np.einsum("kfvp,kfpi,p->kvi", uc[sel], m.N[sel], wf)
        assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(rhs).max()


def test_face_gradient_lifting_keeps_the_jump_mean():
    # eta times the lifting of face f alone, integrated over the face:
    # nsign (S[d, :] / |J|) (sum_j l_j h_j) times the jump's face integral
    m = _box(3, n=3)
    caps = np.random.default_rng(8).integers(0, 3, m.E)
    u = SP.project(m, _state(m, 13), caps)
    _, jmp = _jumps(m, u)
    wf = m.face_weights()
    for q in range(3):
        sel = np.nonzero(caps == q)[0]
        ops = MX.MortarOps(3, q, DG)
        G1 = MX.face_gradients(m, NavierStokes(3, mu=0.01, eta=1.0), sel, ops, u, jmp)
        G0 = MX.face_gradients(m, NavierStokes(3, mu=0.01, eta=0.0), sel, ops, u, jmp)
        S, Jq = MX.metrics(m, sel, ops)
        for d in range(3):
            for s in (0, 1):
                f = 2 * d + s
                lv = ops.ref.lp if s else ops.ref.lm
                h = ops.ref.hp if s else ops.ref.hm
                c = (1.0 if s else -1.0) * float(lv @ h)
                lhs = np.einsum("kvip,p->kvi", G1[:, f] - G0[:, f], wf)
                rhs = c * np.einsum("ki,kv->kvi", S[:, d, :, 0] / Jq[:, :1], jmp[sel, f] @ wf)
                assert np.abs(lhs - rhs).max() <= 1e-12 * max(np.abs(rhs).max(), 1e-300)
