// Host-side FR set-up in double precision: 1D reference operators and the
// curved-element geometry (metric terms, Jacobians, face normals).
#pragma once

#include <cstdint>
#include <vector>

namespace frg {

constexpr int MAXNP = 5;

// 1D ingredients for order p (Np = p+1 Gauss-Legendre points).
struct Ref1D {
    int p = 0, np = 0;
    double x[MAXNP], w[MAXNP];   // GL points and weights
    double gll[MAXNP];           // Gauss-Lobatto points (Np of them)
    double lm[MAXNP], lp[MAXNP]; // l_j(-1), l_j(+1)
    double D[MAXNP][MAXNP];      // l_j'(x_i)
    double hm[MAXNP], hp[MAXNP]; // -g_L'(x_i), g_R'(x_i)
};

// Legendre P_0..P_n and derivatives at x.
void legendre(int n, double x, double* P, double* dP);
void gauss_legendre(int n, double* x, double* w);
void gauss_lobatto(int n, double* x);
double lagrange(const double* xs, int n, int j, double y);
double lagrange_deriv(const double* xs, int n, int j, double y);
// g_L'(x) of the left correction function for degree p (kind 0: DG, 1: Huynh g2)
double corr_left_deriv(int p, int kind, double x);
void build_ref(int p, int kind, Ref1D& r);

// Geometry of one element of order p with geometry order q.
//   nodes [(q+1)^dim][dim]
//   xsp  [Nsp][dim]          solution-point coordinates
//   J    [Nsp]               det(dx/dxi) at solution points
//   S    [dim*dim][Nsp]      |J| dxi_d/dx_i (k = d*dim + i), conservative-curl form
//   Nf   [2*dim][Nfp][dim]   outward area-weighted normals at flux points
void element_geometry(int dim, int q, const Ref1D& r, const double* nodes, double* xsp, double* J,
                      double* S, double* Nf);

// Map x(xi) and dx/dxi at one reference point (for point location).
void element_map(int dim, int q, const double* nodes, const double* xi, double* x, double* A);

}  // namespace frg
