// Host-side FR set-up in double precision (Section 1 FR; Section 3.1 curved
// hexahedra).  Written independently of any test code.
#include "fr_geom.h"

#include <cmath>
#include <cstring>

namespace frg {

void legendre(int n, double x, double* P, double* dP) {
    P[0] = 1.0;
    dP[0] = 0.0;
    if (n == 0) return;
    P[1] = x;
    dP[1] = 1.0;
    for (int k = 1; k < n; ++k) {
        P[k + 1] = ((2 * k + 1) * x * P[k] - k * P[k - 1]) / (k + 1);
        dP[k + 1] = dP[k - 1] + (2 * k + 1) * P[k];
    }
}

void gauss_legendre(int n, double* x, double* w) {
    double P[16], dP[16];
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            legendre(n, z, P, dP);
            const double dz = P[n] / dP[n];
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        legendre(n, z, P, dP);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dP[n] * dP[n]);
    }
    // P_n has definite parity: the roots pair as +-x (0 for odd n) with equal
    // weights; impose it exactly so mirrored operators are bit-symmetric
    for (int i = 0; i < n / 2; ++i) {
        const double a = 0.5 * (x[n - 1 - i] - x[i]);
        const double b = 0.5 * (w[n - 1 - i] + w[i]);
        x[n - 1 - i] = a;
        x[i] = -a;
        w[n - 1 - i] = b;
        w[i] = b;
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

void gauss_lobatto(int n, double* x) {
    // endpoints and the roots of P'_{n-1}; Newton with P''_{N} from the
    // Legendre equation (1 - z^2) P'' = 2 z P' - N (N + 1) P
    const int N = n - 1;
    x[0] = -1.0;
    x[n - 1] = 1.0;
    double P[16], dP[16];
    for (int i = 1; i < N; ++i) {
        double z = -std::cos(M_PI * i / N);
        for (int it = 0; it < 100; ++it) {
            legendre(N, z, P, dP);
            const double d2 = (2.0 * z * dP[N] - N * (N + 1) * P[N]) / (1.0 - z * z);
            const double dz = dP[N] / d2;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = z;
    }
}

double lagrange(const double* xs, int n, int j, double y) {
    double v = 1.0;
    for (int m = 0; m < n; ++m)
        if (m != j) v *= (y - xs[m]) / (xs[j] - xs[m]);
    return v;
}

double lagrange_deriv(const double* xs, int n, int j, double y) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
        if (k == j) continue;
        double t = 1.0 / (xs[j] - xs[k]);
        for (int m = 0; m < n; ++m)
            if (m != j && m != k) t *= (y - xs[m]) / (xs[j] - xs[m]);
        s += t;
    }
    return s;
}

// derivative of the right Radau polynomial R_{R,k} = (-1)^k/2 (P_k - P_{k-1})
static double radau_right_deriv(int k, double x) {
    double P[16], dP[16];
    legendre(k, x, P, dP);
    const double sg = (k % 2 == 0) ? 1.0 : -1.0;
    return 0.5 * sg * (dP[k] - dP[k - 1]);
}

double corr_left_deriv(int p, int kind, double x) {
    const int k = p + 1;
    if (kind == 0) return radau_right_deriv(k, x);
    // Huynh g2 = ((k-1) R_{R,k} + k R_{R,k-1}) / (2k-1)
    return ((k - 1) * radau_right_deriv(k, x) + k * radau_right_deriv(k - 1, x)) / (2.0 * k - 1.0);
}

void build_ref(int p, int kind, Ref1D& r) {
    std::memset(&r, 0, sizeof(r));
    r.p = p;
    r.np = p + 1;
    const int n = r.np;
    gauss_legendre(n, r.x, r.w);
    gauss_lobatto(n, r.gll);
    for (int j = 0; j < n; ++j) {
        r.lm[j] = lagrange(r.x, n, j, -1.0);
        r.lp[j] = lagrange(r.x, n, j, 1.0);
        for (int i = 0; i < n; ++i) r.D[i][j] = lagrange_deriv(r.x, n, j, r.x[i]);
    }
    for (int i = 0; i < n; ++i) {
        r.hm[i] = -corr_left_deriv(p, kind, r.x[i]);
        r.hp[i] = -corr_left_deriv(p, kind, -r.x[i]);
    }
}

// out[m_{dim-1}]..[m_0] = (M_{dim-1} x .. x M_0) in, in [n]..[n] (direction 0 fastest);
// M_d is [m_d][n] row-major.
static void tensor_apply(int dim, int n, const double* in, const double* const* M, const int* m,
                         double* out) {
    if (dim == 2) {
        // t[b][a'] = sum_a M0[a'][a] in[b][a]
        double t[MAXNP * MAXNP];
        for (int b = 0; b < n; ++b)
            for (int a2 = 0; a2 < m[0]; ++a2) {
                double s = 0;
                for (int a = 0; a < n; ++a) s += M[0][a2 * n + a] * in[b * n + a];
                t[b * m[0] + a2] = s;
            }
        for (int b2 = 0; b2 < m[1]; ++b2)
            for (int a2 = 0; a2 < m[0]; ++a2) {
                double s = 0;
                for (int b = 0; b < n; ++b) s += M[1][b2 * n + b] * t[b * m[0] + a2];
                out[b2 * m[0] + a2] = s;
            }
        return;
    }
    double t1[MAXNP * MAXNP * MAXNP], t2[MAXNP * MAXNP * MAXNP];
    for (int c = 0; c < n; ++c)
        for (int b = 0; b < n; ++b)
            for (int a2 = 0; a2 < m[0]; ++a2) {
                double s = 0;
                for (int a = 0; a < n; ++a) s += M[0][a2 * n + a] * in[(c * n + b) * n + a];
                t1[(c * n + b) * m[0] + a2] = s;
            }
    for (int c = 0; c < n; ++c)
        for (int b2 = 0; b2 < m[1]; ++b2)
            for (int a2 = 0; a2 < m[0]; ++a2) {
                double s = 0;
                for (int b = 0; b < n; ++b) s += M[1][b2 * n + b] * t1[(c * n + b) * m[0] + a2];
                t2[(c * m[1] + b2) * m[0] + a2] = s;
            }
    for (int c2 = 0; c2 < m[2]; ++c2)
        for (int b2 = 0; b2 < m[1]; ++b2)
            for (int a2 = 0; a2 < m[0]; ++a2) {
                double s = 0;
                for (int c = 0; c < n; ++c) s += M[2][c2 * n + c] * t2[(c * m[1] + b2) * m[0] + a2];
                out[(c2 * m[1] + b2) * m[0] + a2] = s;
            }
}

// basis matrices [m][n] of the Lagrange polynomials on nodes xs evaluated at ys
static void basis_mat(const double* xs, int n, const double* ys, int m, bool deriv, double* M) {
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j)
            M[i * n + j] = deriv ? lagrange_deriv(xs, n, j, ys[i]) : lagrange(xs, n, j, ys[i]);
}

void element_map(int dim, int q, const double* nodes, const double* xi, double* x, double* A) {
    const int nq = q + 1;
    double xe[3] = {-1.0, 0.0, 1.0};
    if (q == 1) { xe[1] = 1.0; }
    double L[3][3], Ld[3][3];
    for (int d = 0; d < dim; ++d)
        for (int a = 0; a < nq; ++a) {
            L[d][a] = lagrange(xe, nq, a, xi[d]);
            Ld[d][a] = lagrange_deriv(xe, nq, a, xi[d]);
        }
    for (int c = 0; c < dim; ++c) {
        x[c] = 0;
        for (int k = 0; k < dim; ++k) A[c * dim + k] = 0;
    }
    const int nn = (dim == 2) ? nq * nq : nq * nq * nq;
    for (int id = 0; id < nn; ++id) {
        int a[3] = {id % nq, (id / nq) % nq, id / (nq * nq)};
        double w = 1.0;
        for (int d = 0; d < dim; ++d) w *= L[d][a[d]];
        for (int c = 0; c < dim; ++c) x[c] += w * nodes[id * dim + c];
        for (int k = 0; k < dim; ++k) {
            double wk = 1.0;
            for (int d = 0; d < dim; ++d) wk *= (d == k) ? Ld[d][a[d]] : L[d][a[d]];
            for (int c = 0; c < dim; ++c) A[c * dim + k] += wk * nodes[id * dim + c];
        }
    }
}

void element_geometry(int dim, int q, const Ref1D& r, const double* nodes, double* xsp, double* J,
                      double* S, double* Nf) {
    const int n = r.np;
    const int nq = q + 1;
    double xe[3] = {-1.0, 0.0, 1.0};
    if (q == 1) xe[1] = 1.0;
    const int nsp = (dim == 2) ? n * n : n * n * n;
    const int nfp = (dim == 2) ? n : n * n;
    // nodal values on the (q+1)^dim geometry nodes embedded in an n^dim array:
    // first interpolate the map to the GLL grid and to the GL grid.
    double Egll[MAXNP * 3], Edgll[MAXNP * 3], Egl[MAXNP * 3], Edgl[MAXNP * 3];
    basis_mat(xe, nq, r.gll, n, false, Egll);
    basis_mat(xe, nq, r.gll, n, true, Edgll);
    basis_mat(xe, nq, r.x, n, false, Egl);
    basis_mat(xe, nq, r.x, n, true, Edgl);
    // Derivatives of the map and the curl-form products are evaluated from
    // node coordinates relative to the node centroid: a translation changes
    // neither (the Lagrange derivative weights sum to zero; the curl of
    // c grad x_m vanishes for maps inside the interpolation space), and it
    // removes cancellation in elements far from the origin.
    const int nn = (dim == 2) ? nq * nq : nq * nq * nq;
    double cen[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < nn; ++a)
        for (int c = 0; c < dim; ++c) cen[c] += nodes[a * dim + c];
    for (int c = 0; c < dim; ++c) cen[c] /= nn;
    double rnodes[27 * 3];
    for (int a = 0; a < nn; ++a)
        for (int c = 0; c < dim; ++c) rnodes[a * dim + c] = nodes[a * dim + c] - cen[c];
    auto map_eval_of = [&](const double* nd, int comp, const double* M0, const double* M1, const double* M2,
                           double* out) {
        // in: nq^dim node values; matrices [n][nq]; do explicit loops
        if (dim == 2) {
            for (int b2 = 0; b2 < n; ++b2)
                for (int a2 = 0; a2 < n; ++a2) {
                    double s = 0;
                    for (int b = 0; b < nq; ++b)
                        for (int a = 0; a < nq; ++a)
                            s += M1[b2 * nq + b] * M0[a2 * nq + a] * nd[(b * nq + a) * dim + comp];
                    out[b2 * n + a2] = s;
                }
            return;
        }
        for (int c2 = 0; c2 < n; ++c2)
            for (int b2 = 0; b2 < n; ++b2)
                for (int a2 = 0; a2 < n; ++a2) {
                    double s = 0;
                    for (int c = 0; c < nq; ++c)
                        for (int b = 0; b < nq; ++b)
                            for (int a = 0; a < nq; ++a)
                                s += M2[c2 * nq + c] * M1[b2 * nq + b] * M0[a2 * nq + a] *
                                     nd[((c * nq + b) * nq + a) * dim + comp];
                    out[(c2 * n + b2) * n + a2] = s;
                }
    };
    // solution-point coordinates and Jacobian determinant (direct from the map)
    double X[3][MAXNP * MAXNP * MAXNP];
    double A[3][3][MAXNP * MAXNP * MAXNP];  // A[c][k] = dx_c/dxi_k at GL points
    for (int c = 0; c < dim; ++c) {
        map_eval_of(nodes, c, Egl, Egl, Egl, X[c]);
        for (int k = 0; k < dim; ++k)
            map_eval_of(rnodes, c, k == 0 ? Edgl : Egl, k == 1 ? Edgl : Egl, k == 2 ? Edgl : Egl, A[c][k]);
    }
    for (int s = 0; s < nsp; ++s) {
        for (int c = 0; c < dim; ++c) xsp[s * dim + c] = X[c][s];
        if (dim == 2) {
            J[s] = A[0][0][s] * A[1][1][s] - A[0][1][s] * A[1][0][s];
        } else {
            const double a00 = A[0][0][s], a01 = A[0][1][s], a02 = A[0][2][s];
            const double a10 = A[1][0][s], a11 = A[1][1][s], a12 = A[1][2][s];
            const double a20 = A[2][0][s], a21 = A[2][1][s], a22 = A[2][2][s];
            J[s] = a00 * (a11 * a22 - a12 * a21) - a01 * (a10 * a22 - a12 * a20) + a02 * (a10 * a21 - a11 * a20);
        }
    }
    // values of the map and its derivatives on the GLL grid
    double xg[3][MAXNP * MAXNP * MAXNP];
    double ag[3][3][MAXNP * MAXNP * MAXNP];
    for (int c = 0; c < dim; ++c) {
        map_eval_of(rnodes, c, Egll, Egll, Egll, xg[c]);
        for (int k = 0; k < dim; ++k)
            map_eval_of(rnodes, c, k == 0 ? Edgll : Egll, k == 1 ? Edgll : Egll, k == 2 ? Edgll : Egll, ag[c][k]);
    }
    // evaluation of GLL-interpolated fields (and one derivative) on target grids
    double Igl[MAXNP * MAXNP], Dgl[MAXNP * MAXNP];   // GLL -> GL
    basis_mat(r.gll, n, r.x, n, false, Igl);
    basis_mat(r.gll, n, r.x, n, true, Dgl);
    const double ends[2] = {-1.0, 1.0};
    double Iend[2][MAXNP], Dend[2][MAXNP];
    for (int s = 0; s < 2; ++s) {
        basis_mat(r.gll, n, &ends[s], 1, false, Iend[s]);
        basis_mat(r.gll, n, &ends[s], 1, true, Dend[s]);
    }
    // face = -1: volume (GL in every direction); else face index 2d+side
    auto eval = [&](const double* field, int deriv, int face, double* out) {
        const double* M[3];
        int m[3];
        for (int d = 0; d < dim; ++d) {
            const bool at_face = (face >= 0 && (face >> 1) == d);
            if (at_face) {
                const int s = face & 1;
                M[d] = (d == deriv) ? Dend[s] : Iend[s];
                m[d] = 1;
            } else {
                M[d] = (d == deriv) ? Dgl : Igl;
                m[d] = n;
            }
        }
        tensor_apply(dim, n, field, M, m, out);
    };
    // metric terms S[d][i] at a target set (face = -1: solution points)
    auto metrics = [&](int face, double* Sout, int npts) {
        double t1[MAXNP * MAXNP * MAXNP], t2[MAXNP * MAXNP * MAXNP];
        if (dim == 2) {
            // S = [[y_eta, -x_eta], [-y_xi, x_xi]] from the GLL interpolant of the map
            eval(xg[1], 1, face, t1);
            for (int s = 0; s < npts; ++s) Sout[0 * npts + s] = t1[s];
            eval(xg[0], 1, face, t1);
            for (int s = 0; s < npts; ++s) Sout[1 * npts + s] = -t1[s];
            eval(xg[1], 0, face, t1);
            for (int s = 0; s < npts; ++s) Sout[2 * npts + s] = -t1[s];
            eval(xg[0], 0, face, t1);
            for (int s = 0; s < npts; ++s) Sout[3 * npts + s] = t1[s];
            return;
        }
        // S[d][i] = [curl_xi (x_l grad_xi x_m)]_d, (i, l, m) cyclic
        const int ng = n * n * n;
        double w[3][MAXNP * MAXNP * MAXNP];
        for (int i = 0; i < 3; ++i) {
            const int l = (i + 1) % 3, mm = (i + 2) % 3;
            for (int k = 0; k < 3; ++k)
                for (int s = 0; s < ng; ++s) w[k][s] = xg[l][s] * ag[mm][k][s];
            for (int d = 0; d < 3; ++d) {
                const int d1 = (d + 1) % 3, d2 = (d + 2) % 3;
                eval(w[d2], d1, face, t1);
                eval(w[d1], d2, face, t2);
                for (int s = 0; s < npts; ++s) Sout[(d * 3 + i) * npts + s] = t1[s] - t2[s];
            }
        }
    };
    metrics(-1, S, nsp);
    double Sf[9 * MAXNP * MAXNP];
    for (int f = 0; f < 2 * dim; ++f) {
        metrics(f, Sf, nfp);
        const int d = f >> 1;
        const double sg = (f & 1) ? 1.0 : -1.0;
        for (int fp = 0; fp < nfp; ++fp)
            for (int i = 0; i < dim; ++i) Nf[(f * nfp + fp) * dim + i] = sg * Sf[(d * dim + i) * nfp + fp];
    }
}

}  // namespace frg
