// Flux Reconstruction kernels for sm_103a, templated on dimension, order and
// precision.  One warp processes one element (a block holds `epb` warps); the
// element's data are staged in that warp's shared memory with cp.async, every
// operator is applied along lines of solution points, and the phases of a
// kernel are separated by __syncwarp() only.
//
// Per RK stage two sweeps (the two BR2 neighbour dependencies force them):
//   k_visc_face  u, u_f(own, nbr)  -> own-side viscous normal flux at flux points
//   k_residual   u, u_f(own, nbr), viscous fluxes(own, nbr) -> R, fused RK4
//                stage, and the flux-point traces u_f of the stage's output state
// k_traces writes u_f only after the state is set from outside.  Both sweeps
// are compiled per mesh class (metric path, periodic or not; Euler or
// Navier-Stokes for k_residual), so no dead branch of another class stays in
// the kernel.  Smaller kernels: wall forces, surface sampling, volume
// integrals, the energy source of Appendix D, the reduced-degree projection
// and the adaptive time step.
// Notation and steps follow Section 2.1 (Eqs. 1-7) with the FR reading
// described in fr_common.h / fr.h: GL points, DG or g2 correction, Rusanov,
// BR2, metric terms S = |J| dxi/dx in conservative-curl form.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "fr_common.h"

namespace frk {

template <int DIM, int P>
struct Sz {
    static constexpr int NP = P + 1;
    static constexpr int NSP = (DIM == 2) ? NP * NP : NP * NP * NP;
    static constexpr int NFP = (DIM == 2) ? NP : NP * NP;
    static constexpr int NF = 2 * DIM;
    static constexpr int NV = DIM + 2;
};

// Threads per element of the element kernels (k_traces, k_visc_face,
// k_residual): one warp, or two warps for p = 4 in 3D, whose 19 KB of shared
// memory per element would otherwise leave 12 warps per SM to hide latency.
// `lane` below is the thread's index within its element group (0..T-1) and
// the phases of a group are separated by grp_sync (a named barrier per group
// when T = 64; barrier 0 stays free).
template <int DIM, int P>
struct Grp {
    static constexpr int T = (DIM == 3 && P == 4) ? 64 : 32;
};
template <int T>
__device__ __forceinline__ void grp_sync(int grp) {
    if constexpr (T == 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;\n" ::"r"(grp + 1), "n"(T) : "memory");
    }
}

// Face point (side, fp) of the two faces normal to one direction that thread
// `lane` of an element group handles at iteration it; false when it has none.
// One warp per element: t = lane + 32 it runs over side 0, then side 1.  Two
// warps (p = 4 in 3D, 25 points per face, one iteration): the first warp takes
// the 25 points of side 0 and points 0-2 of side 1, the second warp points
// 3-24 of side 1.  The two faces' [v][fp] rows lie 125 floats (29 banks) apart,
// so side-1 points 0-2 use banks 29-31, which side 0 leaves free; points 0-6
// (the plain split) would put two words on each of banks 0-3.
template <int DIM, int P>
__device__ __forceinline__ bool face_pt(int lane, int it, int& side, int& fp) {
    constexpr int T = Grp<DIM, P>::T, NFP = Sz<DIM, P>::NFP;
    if constexpr (T == 64) {
        static_assert(NFP == 25 && Sz<DIM, P>::NV == 5, "the two-warp face split is laid out for p = 4 in 3D");
        side = lane < NFP ? 0 : 1;
        fp = lane < NFP ? lane : lane < 32 ? lane - NFP : lane - 29;
        return lane < 28 || (lane >= 32 && lane < 54);
    } else {
        const int t = lane + T * it;
        side = t >= NFP ? 1 : 0;
        fp = t - side * NFP;
        return t < 2 * NFP;
    }
}

// solution point j (along direction d) of the line through face point fp of a
// face normal to d; face points enumerate the remaining directions in
// increasing order, the lower one fastest
template <int DIM, int NP>
__device__ __forceinline__ int line_sp(int d, int fp, int j) {
    if (DIM == 2) return d == 0 ? j + NP * fp : fp + NP * j;
    const int a = fp % NP, b = fp / NP;
    if (d == 0) return j + NP * (a + NP * b);
    if (d == 1) return a + NP * (j + NP * b);
    return a + NP * (b + NP * j);
}

// inverse of line_sp for direction d: face point and position along the line
template <int DIM, int NP>
__device__ __forceinline__ void sp_split(int sp, int d, int& fp, int& j) {
    if (DIM == 2) {
        const int i0 = sp % NP, i1 = sp / NP;
        if (d == 0) { j = i0; fp = i1; } else { j = i1; fp = i0; }
        return;
    }
    const int i0 = sp % NP, i1 = (sp / NP) % NP, i2 = sp / (NP * NP);
    if (d == 0) { j = i0; fp = i1 + NP * i2; }
    else if (d == 1) { j = i1; fp = i0 + NP * i2; }
    else { j = i2; fp = i0 + NP * i1; }
}

// neighbour face point matching face point fp for orientation code o
// (o = 0, the identity, is the common case: the code is uniform over the
// face, so the branch costs no divergence)
template <int DIM, int NP>
__device__ __forceinline__ int omap(int o, int fp) {
    if (o == 0) return fp;
    if (DIM == 2) return (o & 1) ? NP - 1 - fp : fp;
    int a = fp % NP, b = fp / NP;
    if (o & 4) { const int t = a; a = b; b = t; }
    if (o & 1) a = NP - 1 - a;
    if (o & 2) b = NP - 1 - b;
    return a + NP * b;
}

// ---------------------------------------------------------------- physics
template <int DIM, typename Real>
__device__ __forceinline__ Real pressure(const Real* u, Real gm1) {
    Real m2 = Real(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) m2 += u[1 + i] * u[1 + i];
    return gm1 * (u[DIM + 1] - Real(0.5) * m2 / u[0]);
}

// normal component F_inv(u).n of Eq. 3 for any vector n
template <int DIM, typename Real>
__device__ __forceinline__ void flux_inv_n(const Real* u, Real p, const Real* n, Real* Fn) {
    Real mn = Real(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) mn += u[1 + i] * n[i];
    const Real vn = mn / u[0];
    Fn[0] = mn;
#pragma unroll
    for (int i = 0; i < DIM; ++i) Fn[1 + i] = u[1 + i] * vn + p * n[i];
    Fn[DIM + 1] = (u[DIM + 1] + p) * vn;
}

// Rusanov common flux, area-weighted: F^c.N = |N| [ (F_L + F_R).n/2 - lambda (u_R - u_L)/2 ],
// lambda = max(|V_L.n| + c_L, |V_R.n| + c_R); one reciprocal per state and
// one reciprocal square root for the normal.
template <int DIM, typename Real>
__device__ __forceinline__ void rusanov(const Real* uL, const Real* uR, const Real* N,
                                        Real gamma, Real gm1, Real* F) {
    constexpr int NV = DIM + 2;
    Real a2 = Real(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) a2 += N[i] * N[i];
    const Real ia = rsqrt(a2);
    const Real area = a2 * ia;
    Real n[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) n[i] = N[i] * ia;
    const Real irL = Real(1) / uL[0], irR = Real(1) / uR[0];
    Real mnL = Real(0), mnR = Real(0), m2L = Real(0), m2R = Real(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        mnL += uL[1 + i] * n[i];
        mnR += uR[1 + i] * n[i];
        m2L += uL[1 + i] * uL[1 + i];
        m2R += uR[1 + i] * uR[1 + i];
    }
    const Real pL = gm1 * (uL[NV - 1] - Real(0.5) * m2L * irL);
    const Real pR = gm1 * (uR[NV - 1] - Real(0.5) * m2R * irR);
    const Real vL = mnL * irL, vR = mnR * irR;
    const Real cL = sqrt(gamma * pL * irL), cR = sqrt(gamma * pR * irR);
    const Real lam = fmax(fabs(vL) + cL, fabs(vR) + cR);
    const Real h = Real(0.5) * area;
    const Real hl = h * lam;
    F[0] = h * (mnL + mnR) - hl * (uR[0] - uL[0]);
#pragma unroll
    for (int i = 0; i < DIM; ++i)
        F[1 + i] = h * (uL[1 + i] * vL + uR[1 + i] * vR + (pL + pR) * n[i]) - hl * (uR[1 + i] - uL[1 + i]);
    F[NV - 1] = h * ((uL[NV - 1] + pL) * vL + (uR[NV - 1] + pR) * vR) - hl * (uR[NV - 1] - uL[NV - 1]);
}

// Viscous flux F_vis (Eqs. 4, 6, 7 in the standard sign: [0, tau_ij, V_i tau_ij - q_j],
// q_j = -(mu gamma / Pr) de/dx_j) from u and conserved-variable gradients G[v][j].
template <int DIM, typename Real>
__device__ __forceinline__ void visc_flux(const Real* u, const Real (*G)[DIM], Real mu, Real kappa,
                                          Real (*F)[DIM]) {
    constexpr int NV = DIM + 2;
    const Real ir = Real(1) / u[0];
    Real V[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) V[i] = u[1 + i] * ir;
    Real gV[DIM][DIM];
    Real ge[DIM];
    const Real Er = u[NV - 1] * ir;
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        Real s = (G[NV - 1][j] - Er * G[0][j]) * ir;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            gV[i][j] = (G[1 + i][j] - V[i] * G[0][j]) * ir;
            s -= V[i] * gV[i][j];
        }
        ge[j] = s;
    }
    Real div = Real(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) div += gV[i][i];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        F[0][j] = Real(0);
        Real work = Real(0);
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            Real t = mu * (gV[i][j] + gV[j][i]);
            if (i == j) t -= Real(2.0 / 3.0) * mu * div;
            F[1 + i][j] = t;
            work += V[i] * t;
        }
        F[NV - 1][j] = work + kappa * ge[j];
    }
}

// The same viscous flux contracted with a vector N, F_vis(u, G).N, without
// forming the tensor: (tau N)_i = mu sum_j (dV_i/dx_j + dV_j/dx_i) N_j
// - (2/3) mu div V N_i and the energy entry V.(tau N) - q.N.
template <int DIM, typename Real>
__device__ __forceinline__ void visc_flux_n(const Real* u, const Real (*G)[DIM], Real mu, Real kappa, const Real* N,
                                            Real* Fn) {
    constexpr int NV = DIM + 2;
    const Real ir = Real(1) / u[0];
    Real V[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) V[i] = u[1 + i] * ir;
    Real gV[DIM][DIM];
    Real gn = Real(0);
    const Real Er = u[NV - 1] * ir;
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        Real s = (G[NV - 1][j] - Er * G[0][j]) * ir;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            gV[i][j] = (G[1 + i][j] - V[i] * G[0][j]) * ir;
            s -= V[i] * gV[i][j];
        }
        gn += s * N[j];
    }
    Real div = Real(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) div += gV[i][i];
    const Real c23 = Real(2.0 / 3.0) * mu * div;
    Real en = Real(0);
    Fn[0] = Real(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        Real a = Real(0);
#pragma unroll
        for (int j = 0; j < DIM; ++j) a += (gV[i][j] + gV[j][i]) * N[j];
        const Real tn = mu * a - c23 * N[i];
        Fn[1 + i] = tn;
        en += V[i] * tn;
    }
    Fn[NV - 1] = en + kappa * gn;
}

// visc_flux_n for an area normal along axis d (N = Nd e_d, axis-aligned
// elements): only column d of the flux tensor is formed, the terms that the
// zero components of N would cancel are left out, and the surviving ones keep
// visc_flux_n's order of operations.
template <int DIM, typename Real>
__device__ __forceinline__ void visc_flux_axis(const Real* u, const Real (*G)[DIM], Real mu, Real kappa, int d,
                                               Real Nd, Real* Fn) {
    constexpr int NV = DIM + 2;
    const Real ir = Real(1) / u[0];
    Real V[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) V[i] = u[1 + i] * ir;
    Real gV[DIM][DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int i = 0; i < DIM; ++i) gV[i][j] = (G[1 + i][j] - V[i] * G[0][j]) * ir;
    const Real Er = u[NV - 1] * ir;
    Real s = (G[NV - 1][d] - Er * G[0][d]) * ir;
#pragma unroll
    for (int i = 0; i < DIM; ++i) s -= V[i] * gV[i][d];
    const Real gn = s * Nd;
    Real div = Real(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) div += gV[i][i];
    const Real c23 = Real(2.0 / 3.0) * mu * div;
    Real en = Real(0);
    Fn[0] = Real(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        const Real a = (gV[i][d] + gV[d][i]) * Nd;
        const Real tn = i == d ? mu * a - c23 * Nd : mu * a;
        Fn[1 + i] = tn;
        en += V[i] * tn;
    }
    Fn[NV - 1] = en + kappa * gn;
}

// Rusanov flux for an area normal along axis d (N = Nd e_d): rusanov with the
// zero components of N left out.
template <int DIM, typename Real>
__device__ __forceinline__ void rusanov_axis(const Real* uL, const Real* uR, int d, Real Nd, Real gamma, Real gm1,
                                             Real* F) {
    constexpr int NV = DIM + 2;
    const Real a2 = Nd * Nd;
    const Real ia = rsqrt(a2);
    const Real area = a2 * ia;
    const Real nd = Nd * ia;
    const Real irL = Real(1) / uL[0], irR = Real(1) / uR[0];
    Real m2L = Real(0), m2R = Real(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        m2L += uL[1 + i] * uL[1 + i];
        m2R += uR[1 + i] * uR[1 + i];
    }
    const Real mnL = uL[1 + d] * nd, mnR = uR[1 + d] * nd;
    const Real pL = gm1 * (uL[NV - 1] - Real(0.5) * m2L * irL);
    const Real pR = gm1 * (uR[NV - 1] - Real(0.5) * m2R * irR);
    const Real vL = mnL * irL, vR = mnR * irR;
    const Real cL = sqrt(gamma * pL * irL), cR = sqrt(gamma * pR * irR);
    const Real lam = fmax(fabs(vL) + cL, fabs(vR) + cR);
    const Real h = Real(0.5) * area;
    const Real hl = h * lam;
    F[0] = h * (mnL + mnR) - hl * (uR[0] - uL[0]);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        const Real fl = i == d ? uL[1 + i] * vL + uR[1 + i] * vR + (pL + pR) * nd : uL[1 + i] * vL + uR[1 + i] * vR;
        F[1 + i] = h * fl - hl * (uR[1 + i] - uL[1 + i]);
    }
    F[NV - 1] = h * ((uL[NV - 1] + pL) * vL + (uR[NV - 1] + pR) * vR) - hl * (uR[NV - 1] - uL[NV - 1]);
}

// Boundary states: ghost for the inviscid flux and common solution u_b.
template <int DIM, typename Real>
__device__ __forceinline__ void bc_state(int tag, const Real* uL, const Real* N, const Phys<Real>& ph,
                                         Real* ug, Real* ub) {
    constexpr int NV = DIM + 2;
    Real a2 = Real(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) a2 += N[i] * N[i];
    const Real ia = Real(1) / sqrt(a2);
    Real n[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) n[i] = N[i] * ia;
    if (tag == FR_BC_WALL) {
        if (ph.viscous) {
            Real m2 = Real(0);
            ug[0] = uL[0];
            ub[0] = uL[0];
#pragma unroll
            for (int i = 0; i < DIM; ++i) {
                ug[1 + i] = -uL[1 + i];
                ub[1 + i] = Real(0);
                m2 += uL[1 + i] * uL[1 + i];
            }
            ug[NV - 1] = uL[NV - 1];
            ub[NV - 1] = uL[NV - 1] - Real(0.5) * m2 / uL[0];
        } else {
            Real mn = Real(0);
#pragma unroll
            for (int i = 0; i < DIM; ++i) mn += uL[1 + i] * n[i];
            ug[0] = uL[0];
            ub[0] = uL[0];
#pragma unroll
            for (int i = 0; i < DIM; ++i) {
                ug[1 + i] = uL[1 + i] - Real(2) * mn * n[i];
                ub[1 + i] = uL[1 + i] - mn * n[i];
            }
            ug[NV - 1] = uL[NV - 1];
            ub[NV - 1] = uL[NV - 1] - Real(0.5) * mn * mn / uL[0];
        }
        return;
    }
    // characteristic far field
    const Real g = ph.gamma, gm1 = ph.gm1;
    const Real rhoL = uL[0];
    const Real pL = pressure<DIM>(uL, gm1);
    const Real cL = sqrt(g * pL / rhoL);
    Real vnL = Real(0), vnI = Real(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
        vnL += uL[1 + i] * n[i];
        vnI += ph.vel_inf[i] * n[i];
    }
    vnL /= rhoL;
    const Real cI = sqrt(g * ph.p_inf / ph.rho_inf);
    if (fabs(vnI) >= cI) {
        if (vnI < Real(0)) {
            Real v2 = Real(0);
            ub[0] = ph.rho_inf;
#pragma unroll
            for (int i = 0; i < DIM; ++i) {
                ub[1 + i] = ph.rho_inf * ph.vel_inf[i];
                v2 += ph.vel_inf[i] * ph.vel_inf[i];
            }
            ub[NV - 1] = ph.p_inf / gm1 + Real(0.5) * ph.rho_inf * v2;
        } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) ub[v] = uL[v];
        }
    } else {
        const Real Rp = vnL + Real(2) * cL / gm1;
        const Real Rm = vnI - Real(2) * cI / gm1;
        const Real vnb = Real(0.5) * (Rp + Rm);
        const Real cb = Real(0.25) * gm1 * (Rp - Rm);
        Real s, Vt[DIM];
        if (vnb > Real(0)) {
            s = pL / pow(rhoL, g);
#pragma unroll
            for (int i = 0; i < DIM; ++i) Vt[i] = uL[1 + i] / rhoL - vnL * n[i];
        } else {
            s = ph.p_inf / pow(ph.rho_inf, g);
#pragma unroll
            for (int i = 0; i < DIM; ++i) Vt[i] = ph.vel_inf[i] - vnI * n[i];
        }
        const Real rhob = pow(cb * cb / (g * s), Real(1) / gm1);
        const Real pb = rhob * cb * cb / g;
        Real v2 = Real(0);
        ub[0] = rhob;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            const Real Vb = Vt[i] + vnb * n[i];
            ub[1 + i] = rhob * Vb;
            v2 += Vb * Vb;
        }
        ub[NV - 1] = pb / gm1 + Real(0.5) * rhob * v2;
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) ug[v] = ub[v];
}

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// explicitly rounded arithmetic of the stage updates, so that the classic RK4
// update and the coefficient form with RK4's coefficients round identically
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// Per-element (per-warp) shared-memory footprint of each kernel, in Reals.
// Regions (Reals) of one warp's shared memory.  F = NF*NV*NFP is one
// element's face data, U = NV*NSP its state.
//   visc : A su[U] | B sj[F] | C sl[F] | D sg[max(DIM*U, F)]  (D holds the
//          staged neighbour traces during the face phase; affine meshes need
//          no gradient volume, so there D is [F] only)
//   resid: A su[U] | B sj[max(U,F)] (sd after the gradient) | C sc[F]
//          (staged own viscous fluxes until each entry is replaced by the
//          common flux of the same face point) | D sF[max(DIM*U, 2F)] (own +
//          staged neighbour traces during the face phase) | E staged
//          neighbour viscous fluxes [F] (face phase)
template <int DIM, int P>
struct Smem {
    using Z = Sz<DIM, P>;
    static constexpr int U = Z::NV * Z::NSP;
    static constexpr int F = Z::NF * Z::NV * Z::NFP;
    static constexpr int imax(int a, int b) { return a > b ? a : b; }
    static constexpr int traces = U;
    static constexpr int vB = U, vC = vB + F, vD = vC + F;
    static constexpr int visc = vD + imax(DIM * U, F);
    static constexpr int visc_a = vD + F;   // affine: no gradient volume, region D holds the neighbour traces
    static constexpr int rB = U, rC = rB + imax(U, F), rD = rC + F, rE = rD + imax(DIM * U, 2 * F);
    static constexpr int resid = rE + F;
    // curved meshes also stage the element's S [DIM*DIM][NSP] and 1/|J| [NSP]:
    // in an extra region after visc's, and in resid's region E once the face
    // phase is over
    static constexpr int G = DIM * DIM * Z::NSP + Z::NSP;
    static constexpr int visc_c = visc + G;
    static constexpr int resid_c = rE + imax(F, G);
    // pipelined face kernel on affine meshes: two buffers per element group,
    // each [state U | own traces F | neighbour traces F | S, 1/|J|, normals]
    static constexpr int GEO = (DIM * DIM + 1 + 2 * DIM * DIM + 3) / 4 * 4;
    static constexpr int pl = U, pn = U + F, pg = U + 2 * F;
    static constexpr int visc_buf = (pg + GEO + 3) / 4 * 4;
    static constexpr int visc_p = 2 * visc_buf;
};
template <int DIM, int P, typename Real>
__host__ __device__ constexpr size_t smem_traces(int wpb) { return sizeof(Real) * size_t(wpb) * Smem<DIM, P>::traces; }
template <int DIM, int P, typename Real>
__host__ __device__ constexpr size_t smem_visc(int wpb, bool curved) {
    return sizeof(Real) * size_t(wpb) * (curved ? Smem<DIM, P>::visc_c : Smem<DIM, P>::visc_p);
}
template <int DIM, int P, typename Real>
__host__ __device__ constexpr size_t smem_resid(int wpb, bool curved) {
    return sizeof(Real) * size_t(wpb) * (curved ? Smem<DIM, P>::resid_c : Smem<DIM, P>::resid);
}

template <int DIM, typename Real>
__device__ __forceinline__ void load_normal(const Geo<Real>& g, int64_t e, int f, int fp, Real* N) {
    const Real* p = g.N + (e * (2 * DIM) + f) * g.sN_f + fp * g.sN_fp;
#pragma unroll
    for (int i = 0; i < DIM; ++i) N[i] = p[i];
}

// ------------------------------------------------------------------ warp helpers
// All element kernels below give one warp one element.  Operator entries are
// read from the __grid_constant__ parameter with indices that are
// compile-time after unrolling, so they become constant-bank operands.  The
// xi_d = +1 face uses the mirror symmetry of the GL points: l_j(+1) =
// l_{NP-1-j}(-1) and h_+(x_i) = h_-(x_{NP-1-i}).

// metric terms S[d][i] at solution point sp (affine: one set per element)
template <int DIM, typename Real>
__device__ __forceinline__ void load_S(const Geo<Real>& g, int64_t e, int sp, Real* S) {
#pragma unroll
    for (int k = 0; k < DIM * DIM; ++k) S[k] = g.S[e * g.sS_e + k * g.sS_k + sp * g.sS_sp];
}

// ---- placement of volume data in shared memory
// Volume arrays (state, gradients, fluxes, divergence) hold variables of NSP
// points each; point (i0, i1, i2) of variable v.  For p = 3 in 3D with
// 4-byte reals the 4-point rows are permuted within each variable: row
// (i1, i2) of v sits at row (i1 ^ a, i2 ^ b) with b = v & 1 and
// a = (i2 >> 1) | (b << 1).  Line passes put consecutive variables on lanes
// 0-15 and 16-31, so with this placement the lines of all three directions,
// the point-wise passes (lane = point) and the per-face-point reads each touch
// 32 distinct banks, and every row stays a 16-byte vector along xi_0.
template <int DIM, int P, typename Real>
struct Vol {
    static constexpr int NP = P + 1;
    static constexpr int NSP = Sz<DIM, P>::NSP;
    static constexpr bool SWZ = DIM == 3 && NP == 4 && sizeof(Real) == 4;
    static constexpr bool ROW4 = NP == 4 && sizeof(Real) == 4;  // a row is one float4
    __device__ __forceinline__ static int at(int v, int i0, int i1, int i2) {
        if constexpr (SWZ) {
            const int b = v & 1;
            return v * NSP + 16 * (i2 ^ b) + 4 * (i1 ^ ((i2 >> 1) | (b << 1))) + i0;
        } else {
            return v * NSP + i0 + NP * (i1 + NP * i2);
        }
    }
    // point sp = i0 + NP i1 (+ NP^2 i2) of variable v (in the plain placement
    // simply v NSP + sp, written so that no division by NP is left)
    __device__ __forceinline__ static int pt(int v, int sp) {
        if constexpr (DIM == 2 || !SWZ) return v * NSP + sp;
        else return at(v, sp % NP, (sp / NP) % NP, sp / (NP * NP));
    }
    // point j of the line through face point ln in direction d (see line_sp);
    // in the plain placement lines along xi_0 and xi_2 need no division by NP
    __device__ __forceinline__ static int line(int v, int d, int ln, int j) {
        if constexpr (DIM == 2) {
            return v * NSP + line_sp<DIM, NP>(d, ln, j);
        } else if constexpr (!SWZ) {
            if (d == 0) return v * NSP + NP * ln + j;
            if (d == 2) return v * NSP + ln + NP * NP * j;
            return v * NSP + ln % NP + NP * (j + NP * (ln / NP));
        } else {
            const int a = ln % NP, b = ln / NP;
            if (d == 0) return at(v, j, a, b);
            if (d == 1) return at(v, a, j, b);
            return at(v, a, b, j);
        }
    }
};

// the NP values of line ln (direction d) of variable v; a direction-0 line is
// one contiguous row (a single 16-byte access when a row is a float4)
template <int DIM, int P, typename Real>
__device__ __forceinline__ void vload_line(const Real* X, int v, int d, int ln, Real (&s)[P + 1]) {
    using V = Vol<DIM, P, Real>;
    if constexpr (V::ROW4) {
        if (d == 0) {
            const float4 r = *reinterpret_cast<const float4*>(X + V::line(v, 0, ln, 0));
            s[0] = r.x;
            s[1] = r.y;
            s[2] = r.z;
            s[3] = r.w;
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < P + 1; ++j) s[j] = X[V::line(v, d, ln, j)];
}
template <int DIM, int P, typename Real>
__device__ __forceinline__ void vstore_line(Real* X, int v, int d, int ln, const Real (&s)[P + 1]) {
    using V = Vol<DIM, P, Real>;
    if constexpr (V::ROW4) {
        if (d == 0) {
            *reinterpret_cast<float4*>(X + V::line(v, 0, ln, 0)) = make_float4(s[0], s[1], s[2], s[3]);
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < P + 1; ++j) X[V::line(v, d, ln, j)] = s[j];
}

// The (variable, line) task of a lane at iteration it of a line pass, task
// index t = v NFP + ln.  When NFP divides 32 a lane keeps its line, and the
// parity of its variable, at every iteration: its accesses then use the
// reference variable vref, whose shared offsets depend on the lane only (the
// compiler keeps them out of the loop), in an array shifted by whole
// variables (an even number of them, so the permuted placement is unchanged).
template <int DIM, int P, int T = Grp<DIM, P>::T>
struct LineTask {
    int t, v, ln, vref, shift;
    __device__ __forceinline__ LineTask(int lane, int it) {
        constexpr int NFP = Sz<DIM, P>::NFP, NSP = Sz<DIM, P>::NSP;
        t = lane + T * it;
        if constexpr (T % NFP == 0 && (T / NFP) % 2 == 0) {
            constexpr int VPI = T / NFP;
            vref = lane / NFP;
            ln = lane % NFP;
            v = vref + VPI * it;
            shift = VPI * it * NSP;
        } else {
            v = t / NFP;
            ln = t % NFP;
            vref = v;
            shift = 0;
        }
    }
};

// q[i] += sum_j D[i][j] s[j].  In FP32 the rows go as packed pairs (two FP32
// FMAs per instruction, the same order of operations), an odd last row alone.
template <int NP, typename Real>
__device__ __forceinline__ void apply_D(const Ops<Real>& op, const Real (&s)[NP], Real (&q)[NP]) {
    if constexpr (sizeof(Real) == 4) {
        float2 a[NP / 2];
#pragma unroll
        for (int r = 0; r < NP / 2; ++r) a[r] = make_float2(q[2 * r], q[2 * r + 1]);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            const float2 sj = make_float2(s[j], s[j]);
#pragma unroll
            for (int r = 0; r < NP / 2; ++r)
                a[r] = __ffma2_rn(make_float2(op.D[(2 * r) * MAXNP + j], op.D[(2 * r + 1) * MAXNP + j]), sj, a[r]);
            if constexpr (NP % 2 == 1) q[NP - 1] += op.D[(NP - 1) * MAXNP + j] * s[j];
        }
#pragma unroll
        for (int r = 0; r < NP / 2; ++r) {
            q[2 * r] = a[r].x;
            q[2 * r + 1] = a[r].y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < NP; ++i)
#pragma unroll
            for (int j = 0; j < NP; ++j) q[i] += op.D[i * MAXNP + j] * s[j];
    }
}

// m = sum_j l_j(-1) s_j and p = sum_j l_j(+1) s_j of a line held in
// registers; in FP32 as one packed pair (same order of operations)
template <int NP, typename Real>
__device__ __forceinline__ void ends_of(const Ops<Real>& op, const Real (&s)[NP], Real& m, Real& p) {
    if constexpr (sizeof(Real) == 4) {
        float2 mp = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int j = 0; j < NP; ++j)
            mp = __ffma2_rn(make_float2(op.lm[j], op.lm[NP - 1 - j]), make_float2(s[j], s[j]), mp);
        m = mp.x;
        p = mp.y;
    } else {
        m = Real(0);
        p = Real(0);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            m += op.lm[j] * s[j];
            p += op.lm[NP - 1 - j] * s[j];
        }
    }
}

// ---- line operators on the tensor cores (precision modes FR_TF32_TC and
// FR_BF16X3_TC of the residual kernel).  A pass over the lines of direction d
// takes them 16 at a time as the rows of an m16n8k8 MMA: A[row][k] = point k
// of the row's line (zero past NP), B[k][n] = D[n][k] for n < NP,
// l_k(-1) for n = NP, l_k(+1) for n = NP + 1, zero beyond, so that one MMA
// gives each line's derivative at its NP points and both of its end values,
// accumulated in FP32.  OPM 1: operands rounded to TF32; OPM 2: each operand
// split into two BF16 parts, hi + lo, and three MMAs (hi hi + hi lo + lo hi).
// Fragments of m16n8k8 (g = lane / 4, t = lane % 4 within the warp): TF32 A
// (g, t), (g+8, t), (g, t+4), (g+8, t+4), B (t, g), (t+4, g); BF16 A the
// pairs (g, 2t..2t+1), (g+8, 2t..2t+1), B (2t..2t+1, g); C (g, 2t), (g, 2t+1),
// (g+8, 2t), (g+8, 2t+1).
__device__ __forceinline__ uint32_t tf32_of(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void bf16_split(float x, unsigned short& hi, unsigned short& lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
}
__device__ __forceinline__ uint32_t pack2(unsigned short a, unsigned short b) {
    return uint32_t(a) | (uint32_t(b) << 16);
}
__device__ __forceinline__ void mma_tf32(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(b0));
}

// B[k][n] of the line-operator MMA (see above)
template <int NP>
__device__ __forceinline__ float tc_b(const Ops<float>& op, int k, int n) {
    if (k >= NP) return 0.0f;
    if (n < NP) return op.D[n * MAXNP + k];
    if (n == NP) return op.lm[k];
    if (n == NP + 1) return op.lm[NP - 1 - k];
    return 0.0f;
}

// this thread's B fragment: TF32 {b0, b1}; BF16x3 {hi, lo}
template <int NP, int OPM>
__device__ __forceinline__ void tc_b_frag(const Ops<float>& op, int lw, uint32_t (&bf)[2]) {
    const int g = lw >> 2, t = lw & 3;
    if constexpr (OPM == 1) {
        bf[0] = tf32_of(tc_b<NP>(op, t, g));
        bf[1] = tf32_of(tc_b<NP>(op, t + 4, g));
    } else {
        unsigned short h0, l0, h1, l1;
        bf16_split(tc_b<NP>(op, 2 * t, g), h0, l0);
        bf16_split(tc_b<NP>(op, 2 * t + 1, g), h1, l1);
        bf[0] = pack2(h0, h1);
        bf[1] = pack2(l0, l1);
    }
}

// C of one tile of 16 line tasks, rows r0 = t0 (this thread's g) and r1 = t0 + 8:
// line task t of direction d is (variable vbase + t / NFP, line t % NFP) of X
template <int DIM, int P, int OPM>
__device__ __forceinline__ void tc_tile(const float* X, int vbase, int d, int t0, const uint32_t (&bf)[2], int lw,
                                        float (&c)[4]) {
    using VL = Vol<DIM, P, float>;
    constexpr int NP = P + 1, NFP = Sz<DIM, P>::NFP, NL = Sz<DIM, P>::NV * NFP;
    const int t = lw & 3, t1 = t0 + 8;
    auto x = [&](int row, int k) -> float {
        return (row < NL && k < NP) ? X[VL::line(vbase + row / NFP, d, row % NFP, k)] : 0.0f;
    };
    c[0] = c[1] = c[2] = c[3] = 0.0f;
    if constexpr (OPM == 1) {
        mma_tf32(c, tf32_of(x(t0, t)), tf32_of(x(t1, t)), tf32_of(x(t0, t + 4)), tf32_of(x(t1, t + 4)), bf[0],
                 bf[1]);
    } else {
        unsigned short h00, l00, h01, l01, h10, l10, h11, l11;
        bf16_split(x(t0, 2 * t), h00, l00);
        bf16_split(x(t0, 2 * t + 1), h01, l01);
        bf16_split(x(t1, 2 * t), h10, l10);
        bf16_split(x(t1, 2 * t + 1), h11, l11);
        const uint32_t ah0 = pack2(h00, h01), ah1 = pack2(h10, h11), al0 = pack2(l00, l01), al1 = pack2(l10, l11);
        mma_bf16(c, al0, al1, bf[0]);   // small products first
        mma_bf16(c, ah0, ah1, bf[1]);
        mma_bf16(c, ah0, ah1, bf[0]);
    }
}

// both end values of line ln (direction d) of variable v of volume array X:
// m = sum_j l_j(-1) s_j and p = sum_j l_j(+1) s_j
template <int DIM, int P, typename Real>
__device__ __forceinline__ void line_ends(const Real* X, int v, const Ops<Real>& op, int d, int ln, Real& m,
                                          Real& p) {
    constexpr int NP = P + 1;
    Real s[NP];
    vload_line<DIM, P>(X, v, d, ln, s);
    ends_of<NP>(op, s, m, p);
}

// ---- cp.async staging (global -> shared without registers)
__device__ __forceinline__ void cp_async16(void* s, const void* g) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(s));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* s, const void* g) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(s));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(g), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// copy N Reals g -> s across the warp; 16-byte chunks when VEC (both sides
// 16-byte aligned and N*sizeof(Real) a multiple of 16), else element-wise
template <int N, bool VEC, typename Real>
__device__ __forceinline__ void warp_stage(Real* s, const Real* g, int lane, int T = 32) {
    if constexpr (VEC) {
        constexpr int NC = int(N * sizeof(Real) / 16);
        constexpr int RPC = int(16 / sizeof(Real));
        for (int c = lane; c < NC; c += T) cp_async16(s + c * RPC, g + c * RPC);
    } else {
        for (int c = lane; c < N; c += T) cp_async_small<int(sizeof(Real))>(s + c, g + c);
    }
}

// as warp_stage, choosing 16-byte chunks at run time when the shared side
// allows them (SVEC) and the global address is 16-byte aligned
template <int N, bool SVEC, typename Real>
__device__ __forceinline__ void warp_stage_auto(Real* s, const Real* g, int lane, int T = 32) {
    constexpr bool V = SVEC && (N * sizeof(Real)) % 16 == 0;
    if (V && (reinterpret_cast<uintptr_t>(g) & 15u) == 0)
        warp_stage<N, V>(s, g, lane, T);
    else
        warp_stage<N, false>(s, g, lane, T);
}

// stage one element's state [NV][NSP] (canonical global layout) into the
// volume placement; rows go as 16-byte copies when the global rows are aligned
template <int DIM, int P, typename Real>
__device__ __forceinline__ void warp_stage_vol(Real* s, const Real* g, int lane, int T = 32) {
    using V = Vol<DIM, P, Real>;
    constexpr int NV = DIM + 2, NP = P + 1, NSP = V::NSP;
    if constexpr (V::ROW4) {
        if ((reinterpret_cast<uintptr_t>(g) & 15u) == 0) {
            constexpr int NR = NV * NSP / NP;   // rows
            for (int k = lane; k < NR; k += T) {
                const int v = k / (NSP / NP), r = k % (NSP / NP);
                cp_async16(s + V::at(v, 0, r % NP, r / NP), g + k * NP);
            }
            return;
        }
    }
    for (int k = lane; k < NV * NSP; k += T)
        cp_async_small<int(sizeof(Real))>(s + V::pt(k / NSP, k % NSP), g + k);
}

// trace on face (d, side) at face point fp of variable v of volume array X:
// sum over the line's points j of c[j] X_j, where c holds l_j(-1) (side 0) or
// l_j(+1) (side 1), selected once per face point by face_coefs
template <int DIM, int P, typename Real>
__device__ __forceinline__ void face_coefs(const Ops<Real>& op, int side, Real (&c)[P + 1]) {
#pragma unroll
    for (int j = 0; j < P + 1; ++j) c[j] = side ? op.lm[P - j] : op.lm[j];
}
template <int DIM, int P, typename Real>
__device__ __forceinline__ Real trace_at(const Real* X, int v, int d, int fp, const Real (&c)[P + 1]) {
    Real s[P + 1];
    vload_line<DIM, P>(X, v, d, fp, s);
    Real acc = Real(0);
#pragma unroll
    for (int j = 0; j < P + 1; ++j) acc += c[j] * s[j];
    return acc;
}

// the traces of the NVV variables 0..NVV-1 of X on one face point; in FP32 two
// variables per packed FMA (the same order of operations as trace_at)
template <int DIM, int P, int NVV, typename Real>
__device__ __forceinline__ void traces_at(const Real* X, int d, int fp, const Real (&c)[P + 1], Real (&tr)[NVV]) {
    constexpr int NP = P + 1;
    if constexpr (sizeof(Real) == 4) {
        float2 cc[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) cc[j] = make_float2(c[j], c[j]);
#pragma unroll
        for (int k = 0; k + 1 < NVV; k += 2) {
            Real s0[NP], s1[NP];
            vload_line<DIM, P>(X, k, d, fp, s0);
            vload_line<DIM, P>(X, k + 1, d, fp, s1);
            float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int j = 0; j < NP; ++j) a = __ffma2_rn(cc[j], make_float2(s0[j], s1[j]), a);
            tr[k] = a.x;
            tr[k + 1] = a.y;
        }
        if constexpr (NVV % 2 == 1) tr[NVV - 1] = trace_at<DIM, P>(X, NVV - 1, d, fp, c);
    } else {
#pragma unroll
        for (int k = 0; k < NVV; ++k) tr[k] = trace_at<DIM, P>(X, k, d, fp, c);
    }
}

// traces of the element state su at every flux point -> ufe [NF][NV][NFP]
// (global or shared), one line per task producing both faces of direction d,
// by T threads (lane 0..T-1)
template <int DIM, int P, int T, typename Real>
__device__ __forceinline__ void warp_write_traces(const Real* su, Real* __restrict__ ufe, const Ops<Real>& op,
                                                  int lane) {
    using Z = Sz<DIM, P>;
    constexpr int NFP = Z::NFP, NV = Z::NV;
    constexpr int NL = NV * NFP, NLI = (NL + T - 1) / T;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
#pragma unroll
        for (int it = 0; it < NLI; ++it) {
            const LineTask<DIM, P, T> tk(lane, it);
            if (NL % T != 0 && tk.t >= NL) break;
            Real m, p;
            line_ends<DIM, P>(su + tk.shift, tk.vref, op, d, tk.ln, m, p);
            ufe[2 * d * NV * NFP + tk.t] = m;
            ufe[(2 * d + 1) * NV * NFP + tk.t] = p;
        }
    }
}

// ------------------------------------------------------------------ kernels
// Sweep A (only after the state is set from outside): traces of u.
template <int DIM, int P, typename Real>
__global__ void k_traces(const Real* __restrict__ u, Real* __restrict__ uf, int64_t E,
                         const __grid_constant__ Ops<Real> op) {
    using Z = Sz<DIM, P>;
    constexpr int T = Grp<DIM, P>::T;   // threads per element
    constexpr int NSP = Z::NSP, NFP = Z::NFP, NF = Z::NF, NV = Z::NV;
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x / T, lane = threadIdx.x % T;
    const int64_t e = int64_t(blockIdx.x) * (blockDim.x / T) + warp;
    if (e >= E) return;
    Real* su = reinterpret_cast<Real*>(smem) + warp * Smem<DIM, P>::traces;
    warp_stage_vol<DIM, P>(su, u + e * NV * NSP, lane, T);
    cp_async_commit();
    cp_async_wait<0>();
    grp_sync<T>(warp);
    warp_write_traces<DIM, P, T>(su, uf + e * NF * NV * NFP, op, lane);
}

// Sweep B on affine elements: one element's face phase from its staged data
// (state su, own traces sl, neighbour traces sn, sgeo = S[DIM*DIM], 1/|J|,
// the outward area normals [NF][DIM]), one pass per face point: the jump
// u_c - u_f, the lifted face gradient and the viscous normal flux, all in
// registers.  With constant metrics the trace of (1/|J|) S^T D u is (1/|J|)
// S^T applied to the traces of the reference derivatives: along the face the
// derivatives of the face trace (interpolation to the face and
// differentiation along it commute), across it the derivative of the normal
// line at its end, sum_j l_j'(+-1) u_j.
template <int DIM, int P, typename Real, bool diag, bool BND, bool VS>
__device__ __forceinline__ void visc_faces_affine(const Real* su, const Real* sl, const Real* sn, const Real* sgeo,
                                                  const int (&codes)[2 * DIM], int64_t e, Real* __restrict__ fvn,
                                                  const Ops<Real>& op, const Phys<Real>& ph, int lane) {
    using Z = Sz<DIM, P>;
    constexpr int T = Grp<DIM, P>::T;
    constexpr int NP = Z::NP, NFP = Z::NFP, NF = Z::NF, NV = Z::NV;
    constexpr int NFI = (2 * NFP + T - 1) / T;
    {
        // the element's metrics and normals, staged with its data
        const Real* S = sgeo;
        const Real iJ = sgeo[DIM * DIM];
        Real SJ[DIM * DIM];   // S / |J|, the element's constant dxi_d/dx_i
#pragma unroll
        for (int k2 = 0; k2 < DIM * DIM; ++k2) SJ[k2] = S[k2] * iJ;
        constexpr bool V4 = NP == 4 && sizeof(Real) == 4 && VS;   // a face-trace row is one float4
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
#pragma unroll
            for (int it = 0; it < NFI; ++it) {
                int side, fp;
                if (!face_pt<DIM, P>(lane, it, side, fp)) continue;
                const int f = 2 * d + side;
                const int code = side ? codes[2 * d + 1] : codes[2 * d];  // static register indices
                const Real* N = sgeo + DIM * DIM + 1 + f * DIM;
                // jumps
                Real uL[NV], jv[NV];
                const Real* tf = sl + f * NV * NFP;
#pragma unroll
                for (int v = 0; v < NV; ++v) uL[v] = tf[v * NFP + fp];
                if (!BND || code >= 0) {
                    const Real* un = sn + f * NV * NFP;
                    const int fpn = omap<DIM, NP>(code & 7, fp);
#pragma unroll
                    for (int v = 0; v < NV; ++v) jv[v] = Real(0.5) * (un[v * NFP + fpn] - uL[v]);
                } else {
                    Real ug[NV], uc[NV];
                    bc_state<DIM>(-code, uL, N, ph, ug, uc);
#pragma unroll
                    for (int v = 0; v < NV; ++v) jv[v] = uc[v] - uL[v];
                }
                // reference derivatives at the face point: across the face
                // (normal line of the volume) and along its two directions
                // (rows of D applied to the face trace)
                const int a = fp % NP, b = DIM == 3 ? fp / NP : 0;
                Real q[DIM][NV];
                if constexpr (sizeof(Real) == 4) {
#pragma unroll
                    for (int v = 0; v + 1 < NV; v += 2) {
                        Real l0[NP], l1[NP];
                        vload_line<DIM, P>(su, v, d, fp, l0);
                        vload_line<DIM, P>(su, v + 1, d, fp, l1);
                        float2 qn = make_float2(0.0f, 0.0f), qa = qn, qb = qn;
                        Real r0[NP], r1[NP];
                        if constexpr (V4) {
                            const float4 x0 = *reinterpret_cast<const float4*>(tf + v * NFP + NP * b);
                            const float4 x1 = *reinterpret_cast<const float4*>(tf + (v + 1) * NFP + NP * b);
                            r0[0] = x0.x; r0[1] = x0.y; r0[2] = x0.z; r0[3] = x0.w;
                            r1[0] = x1.x; r1[1] = x1.y; r1[2] = x1.z; r1[3] = x1.w;
                        } else {
#pragma unroll
                            for (int k2 = 0; k2 < NP; ++k2) {
                                r0[k2] = tf[v * NFP + NP * b + k2];
                                r1[k2] = tf[(v + 1) * NFP + NP * b + k2];
                            }
                        }
#pragma unroll
                        for (int k2 = 0; k2 < NP; ++k2) {
                            const Real dn = side ? -op.dlm[NP - 1 - k2] : op.dlm[k2];
                            qn = __ffma2_rn(make_float2(dn, dn), make_float2(l0[k2], l1[k2]), qn);
                            const Real da = op.D[a * MAXNP + k2];
                            qa = __ffma2_rn(make_float2(da, da), make_float2(r0[k2], r1[k2]), qa);
                            if constexpr (DIM == 3) {
                                const Real db = op.D[b * MAXNP + k2];
                                qb = __ffma2_rn(make_float2(db, db),
                                                make_float2(tf[v * NFP + a + k2 * NP], tf[(v + 1) * NFP + a + k2 * NP]),
                                                qb);
                            }
                        }
                        q[d][v] = qn.x;
                        q[d][v + 1] = qn.y;
                        q[d == 0 ? 1 : 0][v] = qa.x;
                        q[d == 0 ? 1 : 0][v + 1] = qa.y;
                        if constexpr (DIM == 3) {
                            q[d == 2 ? 1 : 2][v] = qb.x;
                            q[d == 2 ? 1 : 2][v + 1] = qb.y;
                        }
                    }
                }
#pragma unroll
                for (int v = sizeof(Real) == 4 ? NV - NV % 2 : 0; v < NV; ++v) {
                    Real ln[NP];
                    vload_line<DIM, P>(su, v, d, fp, ln);
                    Real qn = Real(0), qa = Real(0), qb = Real(0);
#pragma unroll
                    for (int k2 = 0; k2 < NP; ++k2) {
                        const Real dn = side ? -op.dlm[NP - 1 - k2] : op.dlm[k2];
                        qn += dn * ln[k2];
                        qa += op.D[a * MAXNP + k2] * tf[v * NFP + NP * b + k2];
                        if constexpr (DIM == 3) qb += op.D[b * MAXNP + k2] * tf[v * NFP + a + k2 * NP];
                    }
                    q[d][v] = qn;
                    q[d == 0 ? 1 : 0][v] = qa;
                    if constexpr (DIM == 3) q[d == 2 ? 1 : 2][v] = qb;
                }
                // lifted physical gradient G = (1/|J|) S^T q + eta lc (u_c - u_f),
                // lc = nsign l(-1).h_-(x) S[d][:] / |J| (the single-face lifting)
                const Real nsg = side ? Real(1) : Real(-1);
                Real G[NV][DIM];
#pragma unroll
                for (int i = 0; i < DIM; ++i) {
                    const Real lci = ph.eta * nsg * op.lhm * SJ[d * DIM + i];
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        Real tr;
                        if constexpr (diag) {
                            tr = SJ[i * DIM + i] * q[i][v];
                        } else {
                            tr = Real(0);
#pragma unroll
                            for (int dd = 0; dd < DIM; ++dd) tr += SJ[dd * DIM + i] * q[dd][v];
                        }
                        // axis-aligned: S[d][i] = 0 for i != d, so is the lifting there
                        G[v][i] = diag && i != d ? tr : tr + lci * jv[v];
                    }
                }
                Real Fn[NV];
                if (!BND || code >= 0) {
                    if constexpr (diag) visc_flux_axis<DIM>(uL, G, ph.mu, ph.kappa, d, N[d], Fn);
                    else visc_flux_n<DIM>(uL, G, ph.mu, ph.kappa, N, Fn);
                } else {
                    Real ug[NV], ub[NV];
                    bc_state<DIM>(-code, uL, N, ph, ug, ub);
                    if constexpr (diag) visc_flux_axis<DIM>(ub, G, ph.mu, ph.kappa, d, N[d], Fn);
                    else visc_flux_n<DIM>(ub, G, ph.mu, ph.kappa, N, Fn);
                    if (code == -FR_BC_WALL) Fn[NV - 1] = Real(0);
                }
                Real* dst = fvn + (e * NF + f) * NV * NFP + fp;
#pragma unroll
                for (int v = 0; v < NV; ++v) dst[v * NFP] = Fn[v];
            }
        }
    }
}

// Sweep B on affine meshes, pipelined: a persistent grid of element groups,
// each walking the elements e0, e0 + G, e0 + 2G, ... (G groups in the grid).
// While a group computes one element's face phase from one shared buffer, the
// cp.async copies of its next element (state, own and neighbour traces,
// metrics, normals) fill the other buffer, so the copy latency overlaps the
// arithmetic; the neighbour codes are read two elements ahead.
template <int DIM, int P, typename Real, int MP, bool BND>
__global__ void k_visc_face_aff(
    const Real* __restrict__ u, const Real* __restrict__ uf, Real* __restrict__ fvn, int64_t E,
    const __grid_constant__ Ops<Real> op, const __grid_constant__ Phys<Real> ph, const __grid_constant__ Geo<Real> g) {
    using Z = Sz<DIM, P>;
    constexpr int T = Grp<DIM, P>::T;   // threads per element
    constexpr int NSP = Z::NSP, NFP = Z::NFP, NF = Z::NF, NV = Z::NV;
    using SM = Smem<DIM, P>;
    constexpr int BUF = SM::visc_buf;
    constexpr int NGEO = DIM * DIM + 1 + NF * DIM;
    static_assert(MP != 0, "affine meshes only");
    constexpr bool VS = (BUF * sizeof(Real)) % 16 == 0 && (NV * NFP * sizeof(Real)) % 16 == 0 &&
                        (SM::pl * sizeof(Real)) % 16 == 0 && (SM::pn * sizeof(Real)) % 16 == 0;
    extern __shared__ __align__(16) unsigned char smem[];
    const int grp = threadIdx.x / T, lane = threadIdx.x % T, lw = lane & 31;
    const int64_t G = int64_t(gridDim.x) * (blockDim.x / T);
    int64_t e = int64_t(blockIdx.x) * (blockDim.x / T) + grp;
    if (e >= E) return;
    Real* const buf = reinterpret_cast<Real*>(smem) + grp * 2 * BUF;
    auto stage = [&](int64_t el, Real* b, int mine) {
        int codes[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) codes[f] = __shfl_sync(0xffffffffu, mine, f);
        if (g.order && g.order[el] < P) return;   // a reduced-degree element (k_red_face)
        warp_stage_vol<DIM, P>(b, u + el * NV * NSP, lane, T);
        warp_stage<NF * NV * NFP, VS>(b + SM::pl, uf + el * NF * NV * NFP, lane, T);
#pragma unroll
        for (int f = 0; f < NF; ++f)
            if (!BND || codes[f] >= 0)
                warp_stage<NV * NFP, VS>(b + SM::pn + f * NV * NFP, uf + int64_t(codes[f] >> 3) * NV * NFP, lane, T);
        for (int k = lane; k < NGEO; k += T) {
            const Real* src = k < DIM * DIM ? g.S + el * g.sS_e + k * g.sS_k
                            : k == DIM * DIM ? g.iJ + el * g.sJ_e
                                             : g.N + (el * NF) * g.sN_f + (k - DIM * DIM - 1);
            cp_async_small<int(sizeof(Real))>(b + SM::pg + k, src);
        }
    };
    int mineA = lw < NF ? g.nbr[e * NF + lw] : 0;                 // codes of e
    int64_t en = e + G;
    int mineB = (en < E && lw < NF) ? g.nbr[en * NF + lw] : 0;   // codes of the next element
    stage(e, buf, mineA);
    cp_async_commit();
    int b = 0;
    for (;;) {
        Real* cur = buf + b * BUF;
        if (en < E) stage(en, buf + (b ^ 1) * BUF, mineB);
        cp_async_commit();
        const int64_t enn = en + G;
        const int mineC = (enn < E && lw < NF) ? g.nbr[enn * NF + lw] : 0;
        cp_async_wait<1>();
        grp_sync<T>(grp);
        int codes[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) codes[f] = __shfl_sync(0xffffffffu, mineA, f);
        if (!g.order || g.order[e] >= P)
            visc_faces_affine<DIM, P, Real, MP == 2, BND, VS>(cur, cur + SM::pl, cur + SM::pn, cur + SM::pg, codes,
                                                              e, fvn, op, ph, lane);
        if (en >= E) break;
        grp_sync<T>(grp);   // every thread is done with cur before it is refilled
        e = en;
        en = enn;
        mineA = mineB;
        mineB = mineC;
        b ^= 1;
    }
}

// Sweep B: BR2 face gradients and the own-side viscous normal flux.  For a
// boundary face the common viscous flux F_vis(u_b, G).N (energy entry zero at
// an adiabatic wall) is written instead.  MP is the mesh's metric path, fixed
// at compile time: 0 per-point metrics (curved), 1 one metric set per element
// (affine), 2 affine with diagonal S (axis-aligned); BND false: the mesh has
// no boundary faces (fully periodic), so the boundary-state code is left out.
template <int DIM, int P, typename Real, int MP, bool BND>
__global__ void __maxnreg__(sizeof(Real) == 4 ? 80 : 168) k_visc_face(const Real* __restrict__ u, const Real* __restrict__ uf, Real* __restrict__ fvn,
                            int64_t E, const __grid_constant__ Ops<Real> op, const __grid_constant__ Phys<Real> ph,
                            const __grid_constant__ Geo<Real> g) {
    using Z = Sz<DIM, P>;
    constexpr int T = Grp<DIM, P>::T;   // threads per element
    constexpr int NP = Z::NP, NSP = Z::NSP, NFP = Z::NFP, NF = Z::NF, NV = Z::NV;
    constexpr int NSPW = (NSP + T - 1) / T;           // solution points per lane
    constexpr int NL = NV * NFP;                    // (variable, line) tasks per direction
    constexpr int NLI = (NL + T - 1) / T;             // ... per lane
    constexpr int NFI = (2 * NFP + T - 1) / T;        // face points of one direction per lane
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x / T, lane = threadIdx.x % T;
    const int64_t e = int64_t(blockIdx.x) * (blockDim.x / T) + warp;
    if (e >= E || (g.order && g.order[e] < P)) return;   // reduced: k_red_*
    using SM = Smem<DIM, P>;
    using VL = Vol<DIM, P, Real>;
    constexpr bool curved = MP == 0;                // per-point metrics, staged after region D
    constexpr bool diag = MP == 2;                  // affine, diagonal S
    Real* su = reinterpret_cast<Real*>(smem) + warp * (curved ? SM::visc_c : SM::visc_a);
    Real* sj = su + SM::vB;              // jumps u_c - u_f   [f][v][fp]
    Real* sl = su + SM::vC;              // own traces u_f    [f][v][fp]
    Real* sg = su + SM::vD;              // gradient          [d or i][v][sp]
    Real* sn = sg;                       // staged neighbour traces [f][v][fp] (face phase only)
    Real* sS = su + SM::visc;            // curved: S [k][sp], 1/|J| [sp]
    // face codes of this element, broadcast to every lane
    int codes[NF];
    {
        const int mine = (lane & 31) < NF ? g.nbr[e * NF + (lane & 31)] : 0;
#pragma unroll
        for (int f = 0; f < NF; ++f) codes[f] = __shfl_sync(0xffffffffu, mine, f);
    }
    // stage the element state, its own and its neighbours' face traces (the
    // traces array holds them for every element) and (curved) the metrics, in
    // three groups
    constexpr bool VW = (SM::visc * sizeof(Real)) % 16 == 0 && (SM::visc_c * sizeof(Real)) % 16 == 0 &&
                        (SM::visc_a * sizeof(Real)) % 16 == 0;
    constexpr bool VS = VW && (NV * NFP * sizeof(Real)) % 16 == 0 && (SM::vD * sizeof(Real)) % 16 == 0 &&
                        (SM::vC * sizeof(Real)) % 16 == 0;
    warp_stage_vol<DIM, P>(su, u + e * NV * NSP, lane, T);
    cp_async_commit();
    warp_stage<NF * NV * NFP, VS>(sl, uf + e * NF * NV * NFP, lane, T);
#pragma unroll
    for (int f = 0; f < NF; ++f)
        if (!BND || codes[f] >= 0)
            warp_stage<NV * NFP, VS>(sn + f * NV * NFP, uf + int64_t(codes[f] >> 3) * NV * NFP, lane, T);
    cp_async_commit();
    if (curved) {
        warp_stage_auto<DIM * DIM * NSP, VW>(sS, g.S + e * g.sS_e, lane, T);
        warp_stage_auto<NSP, VW && ((SM::visc + DIM * DIM * NSP) * sizeof(Real)) % 16 == 0>(
            sS + DIM * DIM * NSP, g.iJ + e * g.sJ_e, lane, T);
    }
    cp_async_commit();
    cp_async_wait<1>();
    grp_sync<T>(warp);
    {
    // B: jumps per face point
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
#pragma unroll
        for (int it = 0; it < NFI; ++it) {
            int side, fp;
            if (!face_pt<DIM, P>(lane, it, side, fp)) continue;
            const int f = 2 * d + side;
            Real uL[NV], uc[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) uL[v] = sl[(f * NV + v) * NFP + fp];
            const int code = side ? codes[2 * d + 1] : codes[2 * d];  // static register indices
            if (!BND || code >= 0) {
                const Real* un = sn + f * NV * NFP;
                const int fpn = omap<DIM, NP>(code & 7, fp);
#pragma unroll
                for (int v = 0; v < NV; ++v) uc[v] = Real(0.5) * (uL[v] + un[v * NFP + fpn]);
            } else {
                Real N[DIM], ug[NV];
                load_normal<DIM>(g, e, f, fp, N);
                bc_state<DIM>(-code, uL, N, ph, ug, uc);
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) sj[(f * NV + v) * NFP + fp] = uc[v] - uL[v];
        }
    }
    grp_sync<T>(warp);  // the gradient below overwrites the staged neighbour traces
    {
        // C1: uncorrected reference gradient along lines: q_d = D_d u
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
#pragma unroll
            for (int it = 0; it < NLI; ++it) {
                const LineTask<DIM, P> tk(lane, it);
                if (NL % T != 0 && tk.t >= NL) break;
                Real s[NP], q[NP];
                vload_line<DIM, P>(su + tk.shift, tk.vref, d, tk.ln, s);
#pragma unroll
                for (int i = 0; i < NP; ++i) q[i] = Real(0);
                apply_D<NP>(op, s, q);
                vstore_line<DIM, P>(sg + tk.shift, d * NV + tk.vref, d, tk.ln, q);
            }
        }
        cp_async_wait<0>();
        grp_sync<T>(warp);
        // C2: physical gradient (1/|J|) S^T q at each solution point, in place
#pragma unroll
        for (int s = 0; s < NSPW; ++s) {
            const int sp = lane + T * s;
            if (NSP % T != 0 && sp >= NSP) break;
            Real q[DIM][NV];
#pragma unroll
            for (int d = 0; d < DIM; ++d)
#pragma unroll
                for (int v = 0; v < NV; ++v) q[d][v] = sg[VL::pt(d * NV + v, sp)];
            Real S[DIM * DIM];
#pragma unroll
            for (int k = 0; k < DIM * DIM; ++k) S[k] = sS[k * NSP + sp];
            const Real iJ = sS[DIM * DIM * NSP + sp];
            if constexpr (sizeof(Real) == 4) {
                // pairs of variables as packed FP32x2 (the same order of operations)
#pragma unroll
                for (int i = 0; i < DIM; ++i)
#pragma unroll
                    for (int v = 0; v + 1 < NV; v += 2) {
                        float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
                        for (int d = 0; d < DIM; ++d)
                            a = __ffma2_rn(make_float2(S[d * DIM + i], S[d * DIM + i]),
                                           make_float2(q[d][v], q[d][v + 1]), a);
                        a = __fmul2_rn(a, make_float2(iJ, iJ));
                        sg[VL::pt(i * NV + v, sp)] = a.x;
                        sg[VL::pt(i * NV + v + 1, sp)] = a.y;
                    }
            }
#pragma unroll
            for (int i = 0; i < DIM; ++i)
#pragma unroll
                for (int v = sizeof(Real) == 4 ? NV - NV % 2 : 0; v < NV; ++v) {
                    Real acc = Real(0);
#pragma unroll
                    for (int d = 0; d < DIM; ++d) acc += S[d * DIM + i] * q[d][v];
                    sg[VL::pt(i * NV + v, sp)] = acc * iJ;
                }
        }
    }
    // normals of this lane's face points, all directions at once
    Real Nr[DIM][NFI][DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
        for (int it = 0; it < NFI; ++it) {
            int side, fp;
            if (face_pt<DIM, P>(lane, it, side, fp)) load_normal<DIM>(g, e, 2 * d + side, fp, Nr[d][it]);
        }
    grp_sync<T>(warp);
    // D: lifted face gradient, viscous normal flux
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
#pragma unroll
        for (int it = 0; it < NFI; ++it) {
            int side, fp;
            if (!face_pt<DIM, P>(lane, it, side, fp)) continue;
            const int f = 2 * d + side;
            const Real nsg = side ? Real(1) : Real(-1);
            Real cf[NP];
            face_coefs<DIM, P>(op, side, cf);
            // lifting coefficient along the line: nsign sum_j l_j h_j S_j[d][i] / J_j
            Real lc[DIM];
            {
#pragma unroll
                for (int i = 0; i < DIM; ++i) lc[i] = Real(0);
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    // point j of the line; weight l(x_j) h(x_j) of its own end
                    const int sp = line_sp<DIM, NP>(d, fp, j);
                    const Real w = side ? op.lm[NP - 1 - j] * op.hm[NP - 1 - j] : op.lm[j] * op.hm[j];
                    const Real c = w * sS[DIM * DIM * NSP + sp];
#pragma unroll
                    for (int i = 0; i < DIM; ++i) lc[i] += c * sS[(d * DIM + i) * NSP + sp];
                }
#pragma unroll
                for (int i = 0; i < DIM; ++i) lc[i] *= nsg;
            }
            Real tr[DIM * NV];   // traces of the physical gradient [i][v]
            traces_at<DIM, P, DIM * NV>(sg, d, fp, cf, tr);
            Real G[NV][DIM];
            Real uL[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const Real jv = sj[(f * NV + v) * NFP + fp];
                uL[v] = sl[(f * NV + v) * NFP + fp];
#pragma unroll
                for (int i = 0; i < DIM; ++i) G[v][i] = tr[i * NV + v] + ph.eta * lc[i] * jv;
            }
            const Real* N = Nr[d][it];
            const int code = side ? codes[2 * d + 1] : codes[2 * d];  // static register indices
            Real Fn[NV];
            if (!BND || code >= 0) {
                visc_flux_n<DIM>(uL, G, ph.mu, ph.kappa, N, Fn);
            } else {
                Real ug[NV], ub[NV];
                bc_state<DIM>(-code, uL, N, ph, ug, ub);
                visc_flux_n<DIM>(ub, G, ph.mu, ph.kappa, N, Fn);
                if (code == -FR_BC_WALL) Fn[NV - 1] = Real(0);
            }
            Real* dst = fvn + (e * NF + f) * NV * NFP + fp;
#pragma unroll
            for (int v = 0; v < NV; ++v) dst[v * NFP] = Fn[v];
        }
    }
    }
}

// Sweep C: common fluxes, corrected gradient, flux divergence with the FR
// correction, R = -(1/|J|)[...], the RK4 stage update and (for the stepping
// stages) the traces of the updated state written for the next stage.  MP and
// BND as for k_visc_face; VISC: Navier-Stokes (BR2 viscous terms) or Euler;
// OPM: the gradient and divergence line operators as FP32 FMAs (0) or on the
// tensor cores with TF32 (1) or BF16x3 (2) operands (float only).  Register
// caps: 96 in FP32 (88 for p = 4 in 3D, 3.6% faster there), 168 in FP64.
template <int DIM, int P, typename Real, int MP, bool VISC, bool BND, int OPM = 0>
__global__ void __maxnreg__(sizeof(Real) == 4 ? (DIM == 3 && P == 4 ? 88 : 96) : 168) k_residual(const Real* __restrict__ u, const Real* __restrict__ uf,
                           const Real* __restrict__ fvn, int64_t E, const __grid_constant__ Ops<Real> op,
                           const __grid_constant__ Phys<Real> ph, const __grid_constant__ Geo<Real> g,
                           const __grid_constant__ Stage<Real> st) {
    using Z = Sz<DIM, P>;
    constexpr int T = Grp<DIM, P>::T;   // threads per element
    constexpr int NP = Z::NP, NSP = Z::NSP, NFP = Z::NFP, NF = Z::NF, NV = Z::NV;
    constexpr int NSPW = (NSP + T - 1) / T;           // solution points per lane
    constexpr int NL = NV * NFP;                    // (variable, line) tasks per direction
    constexpr int NLI = (NL + T - 1) / T;             // ... per lane
    constexpr int NFI = (2 * NFP + T - 1) / T;        // face points of one direction per lane
    constexpr bool PREFETCH = NSPW <= 2;            // RK arrays held in registers
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x / T, lane = threadIdx.x % T;
    const int64_t e = int64_t(blockIdx.x) * (blockDim.x / T) + warp;
    if (e >= E || (g.order && g.order[e] < P)) return;   // reduced: k_red_*
    using SM = Smem<DIM, P>;
    using VL = Vol<DIM, P, Real>;
    constexpr bool curved = MP == 0;                // per-point metrics, staged in region E
    constexpr bool diag = MP == 2;                  // affine, diagonal S
    Real* su = reinterpret_cast<Real*>(smem) + warp * (curved ? SM::resid_c : SM::resid);
    Real* sj = su + SM::rB;              // jumps u_c - u_f      [f][v][fp]
    Real* sd = sj;                       // divergence [v][sp], after the gradient
    Real* sc = su + SM::rC;              // Fc.N - own viscous flux [f][v][fp]
    Real* sF = su + SM::rD;              // own/neighbour traces, q_d, then F~_d  [d][v][sp]
    Real* sl = sF;                       // own traces            [f][v][fp]  (face phase)
    Real* sn = sF + NF * NV * NFP;       // neighbour traces      [f][v][fp]  (face phase)
    Real* so = sc;                       // own viscous fluxes    [f][v][fp]  (face phase)
    Real* sm = su + SM::rE;              // neighbour viscous fluxes [f][v][fp] (face phase)
    Real* sg = sm;                       // curved: S [k][sp], 1/|J| [sp] (after the face phase)
    const int64_t base = e * NV * NSP;
    int codes[NF];
    {
        const int mine = (lane & 31) < NF ? g.nbr[e * NF + (lane & 31)] : 0;
#pragma unroll
        for (int f = 0; f < NF; ++f) codes[f] = __shfl_sync(0xffffffffu, mine, f);
    }
    constexpr bool VW = (SM::resid * sizeof(Real)) % 16 == 0 && (SM::resid_c * sizeof(Real)) % 16 == 0;
    constexpr bool VS = VW && (NV * NFP * sizeof(Real)) % 16 == 0 && (SM::rC * sizeof(Real)) % 16 == 0 &&
                        (SM::rD * sizeof(Real)) % 16 == 0 && (SM::rE * sizeof(Real)) % 16 == 0;
    warp_stage_vol<DIM, P>(su, u + base, lane, T);
    cp_async_commit();
    warp_stage<NF * NV * NFP, VS>(sl, uf + e * NF * NV * NFP, lane, T);
#pragma unroll
    for (int f = 0; f < NF; ++f)
        if (!BND || codes[f] >= 0) {
            warp_stage<NV * NFP, VS>(sn + f * NV * NFP, uf + int64_t(codes[f] >> 3) * NV * NFP, lane, T);
            if constexpr (VISC)
                warp_stage<NV * NFP, VS>(sm + f * NV * NFP, fvn + int64_t(codes[f] >> 3) * NV * NFP, lane, T);
        }
    if constexpr (VISC) warp_stage<NF * NV * NFP, VS>(so, fvn + e * NF * NV * NFP, lane, T);
    cp_async_commit();
    // face normals of this lane's face points, and the RK stage arrays (needed
    // only at the end): issue their loads now
    Real Nr[DIM][NFI][DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
        for (int it = 0; it < NFI; ++it) {
            int side, fp;
            if (face_pt<DIM, P>(lane, it, side, fp)) load_normal<DIM>(g, e, 2 * d + side, fp, Nr[d][it]);
        }
    Real pu0[NSPW][NV], pacc[NSPW][NV];
    if constexpr (PREFETCH) {
        if (st.stage >= 2) {
#pragma unroll
            for (int s = 0; s < NSPW; ++s) {
                const int sp = lane + T * s;
                if (sp < NSP)
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        pu0[s][v] = st.u0[base + v * NSP + sp];
                        pacc[s][v] = st.acc[base + v * NSP + sp];
                    }
            }
        }
    }
    cp_async_wait<0>();
    grp_sync<T>(warp);
    // B: common normal flux (Rusanov minus common viscous) and jumps
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
#pragma unroll
        for (int it = 0; it < NFI; ++it) {
            int side, fp;
            if (!face_pt<DIM, P>(lane, it, side, fp)) continue;
            const int f = 2 * d + side;
            Real uL[NV], uR[NV], uc[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) uL[v] = sl[(f * NV + v) * NFP + fp];
            const Real* N = Nr[d][it];
            const int code = side ? codes[2 * d + 1] : codes[2 * d];  // static register indices
            int fpn = 0;
            if (!BND || code >= 0) {
                fpn = omap<DIM, NP>(code & 7, fp);
                const Real* un = sn + f * NV * NFP;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    uR[v] = un[v * NFP + fpn];
                    uc[v] = Real(0.5) * (uL[v] + uR[v]);
                }
            } else {
                bc_state<DIM>(-code, uL, N, ph, uR, uc);
            }
            Real Fc[NV];
            if constexpr (diag) rusanov_axis<DIM>(uL, uR, d, N[d], ph.gamma, ph.gm1, Fc);
            else rusanov<DIM>(uL, uR, N, ph.gamma, ph.gm1, Fc);
            if constexpr (VISC) {
                const Real* own = so + f * NV * NFP + fp;
                if (!BND || code >= 0) {
                    const Real* nb = sm + f * NV * NFP + fpn;
#pragma unroll
                    for (int v = 0; v < NV; ++v) Fc[v] -= Real(0.5) * (own[v * NFP] - nb[v * NFP]);
                } else {
#pragma unroll
                    for (int v = 0; v < NV; ++v) Fc[v] -= own[v * NFP];
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                sj[(f * NV + v) * NFP + fp] = uc[v] - uL[v];
                sc[(f * NV + v) * NFP + fp] = Fc[v];
            }
        }
    }
    grp_sync<T>(warp);
    // curved meshes: stage S and 1/|J| into region E (free after the face
    // phase); the copy overlaps the gradient pass
    if (curved) {
        warp_stage_auto<DIM * DIM * NSP, VW && (SM::rE * sizeof(Real)) % 16 == 0>(sg, g.S + e * g.sS_e, lane, T);
        warp_stage_auto<NSP, VW && ((SM::rE + DIM * DIM * NSP) * sizeof(Real)) % 16 == 0>(
            sg + DIM * DIM * NSP, g.iJ + e * g.sJ_e, lane, T);
        cp_async_commit();
    }
    // tensor-core mode: this thread's B fragment of the line operators, and
    // its place in the MMA tiles (warp wg of the element group, g, t)
    static_assert(OPM == 0 || sizeof(Real) == 4, "tensor-core line operators take float data");
    constexpr int NTILE = (NL + 15) / 16, NWG = T / 32;
    const int lw = lane & 31, wg = lane >> 5, gq = lw >> 2, tq = lw & 3;
    uint32_t bfr[2] = {0u, 0u};
    if constexpr (OPM != 0) tc_b_frag<NP, OPM>(reinterpret_cast<const Ops<float>&>(op), lw, bfr);
    // C1 (viscous): corrected reference gradient along lines,
    // q_d = D_d u + nsign h_f (u_c - u_f) for the two faces normal to d
    if constexpr (VISC && OPM != 0) {
#pragma unroll 1
        for (int d = 0; d < DIM; ++d)
            for (int q = wg; q < NTILE; q += NWG) {
                float c[4];
                tc_tile<DIM, P, OPM>(reinterpret_cast<const float*>(su), 0, d, 16 * q + gq, bfr, lw, c);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int tt = 16 * q + gq + 8 * h;
                    if (tt >= NL) continue;
                    const int v = tt / NFP, ln = tt % NFP;
                    const Real jL = sj[2 * d * NV * NFP + tt], jR = sj[(2 * d + 1) * NV * NFP + tt];
#pragma unroll
                    for (int w = 0; w < 2; ++w) {
                        const int n = 2 * tq + w;
                        if (n >= NP) continue;
                        sF[VL::line(d * NV + v, d, ln, n)] = c[2 * h + w] + op.hm[NP - 1 - n] * jR - op.hm[n] * jL;
                    }
                }
            }
    }
    if constexpr (VISC && OPM == 0) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
#pragma unroll
            for (int it = 0; it < NLI; ++it) {
                const LineTask<DIM, P> tk(lane, it);
                if (NL % T != 0 && tk.t >= NL) break;
                Real s[NP], q[NP];
                vload_line<DIM, P>(su + tk.shift, tk.vref, d, tk.ln, s);
                const Real jL = sj[2 * d * NV * NFP + tk.t];
                const Real jR = sj[(2 * d + 1) * NV * NFP + tk.t];
#pragma unroll
                for (int i = 0; i < NP; ++i) q[i] = op.hm[NP - 1 - i] * jR - op.hm[i] * jL;
                apply_D<NP>(op, s, q);
                vstore_line<DIM, P>(sF + tk.shift, d * NV + tk.vref, d, tk.ln, q);
            }
        }
    }
    if (curved) cp_async_wait<0>();
    grp_sync<T>(warp);
    // C2: flux at solution points, F~_d = sum_i S[d][i] (F_inv - F_vis)_i
#pragma unroll 1
    for (int s = 0; s < NSPW; ++s) {
        const int sp = lane + T * s;
        if (NSP % T != 0 && sp >= NSP) break;
        Real uu[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) uu[v] = su[VL::pt(v, sp)];
        Real S[DIM * DIM];
        if (curved) {
#pragma unroll
            for (int k = 0; k < DIM * DIM; ++k) S[k] = sg[k * NSP + sp];
        } else {
            load_S<DIM>(g, e, 0, S);
        }
        Real F[NV][DIM];
        const Real ir = Real(1) / uu[0];
        Real m2 = Real(0);
#pragma unroll
        for (int i = 0; i < DIM; ++i) m2 += uu[1 + i] * uu[1 + i];
        const Real p = ph.gm1 * (uu[NV - 1] - Real(0.5) * m2 * ir);
#pragma unroll
        for (int j = 0; j < DIM; ++j) {
            const Real vj = uu[1 + j] * ir;
            F[0][j] = uu[1 + j];
#pragma unroll
            for (int i = 0; i < DIM; ++i) F[1 + i][j] = uu[1 + i] * vj + (i == j ? p : Real(0));
            F[NV - 1][j] = (uu[NV - 1] + p) * vj;
        }
        if constexpr (VISC) {
            const Real iJ = curved ? sg[DIM * DIM * NSP + sp] : g.iJ[e * g.sJ_e];
            Real G[NV][DIM];
            if constexpr (diag) {
#pragma unroll
                for (int v = 0; v < NV; ++v)
#pragma unroll
                    for (int i = 0; i < DIM; ++i) G[v][i] = S[i * DIM + i] * sF[VL::pt(i * NV + v, sp)] * iJ;
            } else {
                if constexpr (sizeof(Real) == 4) {
#pragma unroll
                    for (int v = 0; v + 1 < NV; v += 2)
#pragma unroll
                        for (int i = 0; i < DIM; ++i) {
                            float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
                            for (int d = 0; d < DIM; ++d)
                                a = __ffma2_rn(make_float2(S[d * DIM + i], S[d * DIM + i]),
                                               make_float2(sF[VL::pt(d * NV + v, sp)], sF[VL::pt(d * NV + v + 1, sp)]), a);
                            a = __fmul2_rn(a, make_float2(iJ, iJ));
                            G[v][i] = a.x;
                            G[v + 1][i] = a.y;
                        }
                }
#pragma unroll
                for (int v = sizeof(Real) == 4 ? NV - NV % 2 : 0; v < NV; ++v)
#pragma unroll
                    for (int i = 0; i < DIM; ++i) {
                        Real acc = Real(0);
#pragma unroll
                        for (int d = 0; d < DIM; ++d) acc += S[d * DIM + i] * sF[VL::pt(d * NV + v, sp)];
                        G[v][i] = acc * iJ;
                    }
            }
            Real Fv[NV][DIM];
            visc_flux<DIM>(uu, G, ph.mu, ph.kappa, Fv);
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int i = 0; i < DIM; ++i) F[v][i] -= Fv[v][i];
        }
        if constexpr (diag) {
#pragma unroll
            for (int d = 0; d < DIM; ++d)
#pragma unroll
                for (int v = 0; v < NV; ++v) sF[VL::pt(d * NV + v, sp)] = S[d * DIM + d] * F[v][d];
        } else {
            if constexpr (sizeof(Real) == 4) {
#pragma unroll
                for (int d = 0; d < DIM; ++d)
#pragma unroll
                    for (int v = 0; v + 1 < NV; v += 2) {
                        float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
                        for (int i = 0; i < DIM; ++i)
                            a = __ffma2_rn(make_float2(S[d * DIM + i], S[d * DIM + i]),
                                           make_float2(F[v][i], F[v + 1][i]), a);
                        sF[VL::pt(d * NV + v, sp)] = a.x;
                        sF[VL::pt(d * NV + v + 1, sp)] = a.y;
                    }
            }
#pragma unroll
            for (int d = 0; d < DIM; ++d)
#pragma unroll
                for (int v = sizeof(Real) == 4 ? NV - NV % 2 : 0; v < NV; ++v) {
                    Real acc = Real(0);
#pragma unroll
                    for (int i = 0; i < DIM; ++i) acc += S[d * DIM + i] * F[v][i];
                    sF[VL::pt(d * NV + v, sp)] = acc;
                }
        }
    }
    grp_sync<T>(warp);
    // D+E: per line of direction d, the flux jumps at both ends,
    // Fc.N - nsign I_f[F~_d], and the divergence plus correction, accumulated
    // direction by direction
    if constexpr (OPM != 0) {
#pragma unroll 1
        for (int d = 0; d < DIM; ++d) {
            for (int q = wg; q < NTILE; q += NWG) {
                float c[4];
                tc_tile<DIM, P, OPM>(reinterpret_cast<const float*>(sF), d * NV, d, 16 * q + gq, bfr, lw, c);
                // both end values of rows g and g + 8, from the lanes of the
                // quad that hold columns NP and NP + 1
                const int qb = lw & ~3;
                const float m0 = __shfl_sync(0xffffffffu, NP % 2 == 0 ? c[0] : c[1], qb + NP / 2);
                const float m1 = __shfl_sync(0xffffffffu, NP % 2 == 0 ? c[2] : c[3], qb + NP / 2);
                const float p0 = __shfl_sync(0xffffffffu, (NP + 1) % 2 == 0 ? c[0] : c[1], qb + (NP + 1) / 2);
                const float p1 = __shfl_sync(0xffffffffu, (NP + 1) % 2 == 0 ? c[2] : c[3], qb + (NP + 1) / 2);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int tt = 16 * q + gq + 8 * h;
                    if (tt >= NL) continue;
                    const int v = tt / NFP, ln = tt % NFP;
                    const Real cL = sc[2 * d * NV * NFP + tt] + (h ? m1 : m0);
                    const Real cR = sc[(2 * d + 1) * NV * NFP + tt] - (h ? p1 : p0);
#pragma unroll
                    for (int w = 0; w < 2; ++w) {
                        const int n = 2 * tq + w;
                        if (n >= NP) continue;
                        Real val = op.hm[n] * cL + op.hm[NP - 1 - n] * cR + c[2 * h + w];
                        const int a = VL::line(v, d, ln, n);
                        if (d > 0) val += sd[a];
                        sd[a] = val;
                    }
                }
            }
            grp_sync<T>(warp);
        }
    } else {
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
#pragma unroll
        for (int it = 0; it < NLI; ++it) {
            const LineTask<DIM, P> tk(lane, it);
            if (NL % T != 0 && tk.t >= NL) break;
            Real s[NP];
            vload_line<DIM, P>(sF + tk.shift, d * NV + tk.vref, d, tk.ln, s);
            Real m, pp;
            ends_of<NP>(op, s, m, pp);
            const Real cL = sc[2 * d * NV * NFP + tk.t] + m;
            const Real cR = sc[(2 * d + 1) * NV * NFP + tk.t] - pp;
            Real val[NP];
#pragma unroll
            for (int i = 0; i < NP; ++i) val[i] = op.hm[i] * cL + op.hm[NP - 1 - i] * cR;
            apply_D<NP>(op, s, val);
            if (d > 0) {
                Real prev[NP];
                vload_line<DIM, P>(sd + tk.shift, tk.vref, d, tk.ln, prev);
#pragma unroll
                for (int i = 0; i < NP; ++i) val[i] += prev[i];
            }
            vstore_line<DIM, P>(sd + tk.shift, tk.vref, d, tk.ln, val);
        }
        grp_sync<T>(warp);
    }
    }
    // F: residual and RK stage per solution point; the new stage state
    // replaces su for the traces
    const Real dt = st.dte ? st.dte[e] : st.dt;
    bool bad = false;   // the last stage's new state holds a NaN or an infinity
    // one loop over this lane's values per kind of stage (the stage is uniform
    // over the launch, so only one loop body runs): upd(r, u, u0, acc, gi)
    // stores the stage arrays and returns the new stage state
    auto stage_loop = [&](auto upd) {
#pragma unroll
        for (int s = 0; s < NSPW; ++s) {
            const int sp = lane + T * s;
            if (NSP % T != 0 && sp >= NSP) break;
            const Real iJ = curved ? sg[DIM * DIM * NSP + sp] : g.iJ[e * g.sJ_e];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const int k = VL::pt(v, sp);
                const Real r = -sd[k] * iJ;
                const int64_t gi = base + v * NSP + sp;
                Real u0v = Real(0), accv = Real(0);
                if (st.stage >= 2) {
                    if constexpr (PREFETCH) {
                        u0v = pu0[s][v];
                        accv = pacc[s][v];
                    } else {
                        u0v = st.u0[gi];
                        accv = st.acc[gi];
                    }
                }
                su[k] = upd(r, su[k], u0v, accv, gi);
            }
        }
    };
    if (st.ls) {
        // coefficient form (see Stage); at stage 1 the input is u0 and acc is 0
        const Real fdt = st.cf * dt, cdt = st.cc * dt;
        if (st.last) {
            stage_loop([&](Real r, Real u, Real u0v, Real accv, int64_t gi) {
                if (st.stage == 1) u0v = u;
                const Real an = st.stage == 1 ? mul_rn(fdt, r) : fma_rn(fdt, r, mul_rn(st.ce, accv));
                Real nu = fma_rn(st.cd, an, mul_rn(st.ca, u0v));
                nu = fma_rn(cdt, r, fma_rn(st.cb, u, nu));
                st.u0[gi] = nu;
                bad = bad || not_finite(nu);
                return nu;
            });
        } else {
            stage_loop([&](Real r, Real u, Real u0v, Real accv, int64_t gi) {
                if (st.stage == 1) u0v = u;
                const Real an = st.stage == 1 ? mul_rn(fdt, r) : fma_rn(fdt, r, mul_rn(st.ce, accv));
                Real nu = fma_rn(st.cd, an, mul_rn(st.ca, u0v));
                nu = fma_rn(cdt, r, fma_rn(st.cb, u, nu));
                st.acc[gi] = an;
                st.us[gi] = nu;
                return nu;
            });
        }
    } else {
        switch (st.stage) {
            case 0:
                stage_loop([&](Real r, Real u, Real, Real, int64_t gi) {
                    st.R[gi] = r;
                    return u;
                });
                break;
            case 1:
                stage_loop([&](Real r, Real u, Real, Real, int64_t gi) {
                    st.acc[gi] = mul_rn(dt * Real(1.0 / 6.0), r);
                    const Real nu = fma_rn(dt * Real(0.5), r, u);
                    st.us[gi] = nu;
                    return nu;
                });
                break;
            case 2:
                stage_loop([&](Real r, Real, Real u0v, Real accv, int64_t gi) {
                    st.acc[gi] = fma_rn(dt * Real(1.0 / 3.0), r, accv);
                    const Real nu = fma_rn(dt * Real(0.5), r, u0v);
                    st.us[gi] = nu;
                    return nu;
                });
                break;
            case 3:
                stage_loop([&](Real r, Real, Real u0v, Real accv, int64_t gi) {
                    st.acc[gi] = fma_rn(dt * Real(1.0 / 3.0), r, accv);
                    const Real nu = fma_rn(dt, r, u0v);
                    st.us[gi] = nu;
                    return nu;
                });
                break;
            default:
                stage_loop([&](Real r, Real, Real u0v, Real accv, int64_t gi) {
                    const Real nu = fma_rn(dt * Real(1.0 / 6.0), r, add_rn(u0v, accv));
                    st.u0[gi] = nu;
                    bad = bad || not_finite(nu);
                    return nu;
                });
                break;
        }
    }
    if (st.nonfinite && __any_sync(0xffffffffu, bad) && (lane & 31) == 0) {
        int c = 0;
        while (c + 1 < st.ncand && e >= st.cand_off[c + 1]) ++c;
        atomicOr(st.nonfinite + c, 1);
    }
    if (st.uf_next) {
        grp_sync<T>(warp);
        warp_write_traces<DIM, P, T>(su, st.uf_next + e * NF * NV * NFP, op, lane);
    }
}

// Energy source of Appendix D (Eq. D.1), applied after the residual kernel of
// a stage to the few elements that carry one (warp per source entry).  The
// stage update is linear in the residual, so adding the source's share to the
// stage arrays afterwards equals adding it to R first: stage 0 adds s to R;
// RK4 stages 1-4 add (dt/2, dt/2, dt, dt/6) s to the stage output (us, us,
// us, u0) and (dt/6, dt/3, dt/3, -) s to acc (the coefficient form: (c + d f)
// dt s and f dt s); the element's next traces are then rewritten from its
// updated stage output.
template <int DIM, int P, typename Real>
__global__ void k_source_stage(const __grid_constant__ Src<Real> src, const __grid_constant__ Stage<Real> st,
                               const __grid_constant__ Ops<Real> op) {
    using Z = Sz<DIM, P>;
    constexpr int NSP = Z::NSP, NFP = Z::NFP, NF = Z::NF, NV = Z::NV;
    using VL = Vol<DIM, P, Real>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + warp;
    if (j >= src.nentry) return;
    Real* sst = reinterpret_cast<Real*>(smem) + warp * NV * NSP;   // updated element state (volume placement)
    const int64_t e = src.elem[j];
    const int c = src.cand[j];
    const double dt = double(st.dte ? st.dte[e] : st.dt);
    const double t = src.tnow[c] + src.cfac * dt;
    double amp[MAXSRC];
#pragma unroll
    for (int m = 0; m < MAXSRC; ++m) {
        const double a = src.A[c * MAXSRC + m];
        amp[m] = a != 0.0 ? a * sinpi(2.0 * src.f[c * MAXSRC + m] * t) : 0.0;
    }
    // share of the source in the stage output and in acc: classic RK4, or the
    // coefficient form (acc gains f dt s, the output (c + d f) dt s)
    const bool last = st.ls ? st.last != 0 : st.stage == 4;
    const double cs = st.ls ? (double(st.cc) + double(st.cd) * double(st.cf)) * dt
                            : st.stage == 3 ? dt : st.stage == 4 ? dt / 6.0 : 0.5 * dt;
    const double ca = st.ls ? double(st.cf) * dt : st.stage == 1 ? dt / 6.0 : dt / 3.0;
    const int64_t gbase = (e * NV + (NV - 1)) * NSP;                             // energy row
    for (int sp = lane; sp < NSP; sp += 32) {
        double sv = 0.0;
#pragma unroll
        for (int m = 0; m < MAXSRC; ++m) sv += amp[m] * double(src.w[(int64_t(j) * MAXSRC + m) * NSP + sp]);
        if (st.stage == 0) {
            st.R[gbase + sp] += Real(sv);
            continue;
        }
        const Real du = Real(cs * sv);
        if (last) {
            st.u0[gbase + sp] += du;
        } else {
            st.us[gbase + sp] += du;
            st.acc[gbase + sp] += Real(ca * sv);
        }
    }
    if (st.stage == 0 || !st.uf_next) return;
    __syncwarp();
    // the next traces of this element, rewritten from its updated state with
    // the same line-end arithmetic as every other element's, so that traces
    // always equal the traces of the state (a state set from outside gets the
    // same values bit for bit)
    const Real* out = (last ? st.u0 : st.us) + e * NV * NSP;
    for (int k = lane; k < NV * NSP; k += 32) sst[VL::pt(k / NSP, k % NSP)] = out[k];
    __syncwarp();
    Real* uf = st.uf_next + e * NF * NV * NFP;
#pragma unroll
    for (int d = 0; d < DIM; ++d)
        for (int t = lane; t < NV * NFP; t += 32) {
            Real m, p;
            line_ends<DIM, P>(sst, t / NFP, op, d, t % NFP, m, p);
            uf[2 * d * NV * NFP + t] = m;
            uf[(2 * d + 1) * NV * NFP + t] = p;
        }
}

// Variable polynomial order (Section 3.1, sponge zones), after the residual
// and source kernels of a stage, warp per listed element.  The tensor-product
// projection onto degree q is the 1D projection pm[q] along each direction in
// turn; each line of a direction is read and rewritten by one task, so the
// passes work in place on the staged element.  Arrays a and b (when given) are
// staged together, projected, and written back; the traces of the projected a
// go to uf_out when given.  The stage update is linear in R and the stage's
// inputs already lie in the space, so projecting the stage outputs equals
// projecting R first.
template <int DIM, int P, typename Real>
__global__ void k_sponge(const __grid_constant__ Sponge<Real> sp, Real* __restrict__ a, Real* __restrict__ b,
                         Real* __restrict__ uf_out, const __grid_constant__ Ops<Real> op) {
    using Z = Sz<DIM, P>;
    constexpr int NSP = Z::NSP, NFP = Z::NFP, NF = Z::NF, NV = Z::NV, NP = P + 1;
    constexpr int NL = NV * NFP;
    using VL = Vol<DIM, P, Real>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = blockIdx.x * (blockDim.x >> 5) + warp;
    if (j >= sp.n) return;
    const int64_t e = sp.elem[j];
    const int q = sp.cap[j];
    Real pq[NP][NP];
#pragma unroll
    for (int i = 0; i < NP; ++i)
#pragma unroll
        for (int k = 0; k < NP; ++k) pq[i][k] = sp.pm[q][i * MAXNP + k];
    Real* sa = reinterpret_cast<Real*>(smem) + warp * 2 * NV * NSP;
    Real* sb = sa + NV * NSP;
    const int narr = b ? 2 : 1;
    warp_stage_vol<DIM, P>(sa, a + e * NV * NSP, lane);
    if (b) warp_stage_vol<DIM, P>(sb, b + e * NV * NSP, lane);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
#pragma unroll 1
    for (int arr = 0; arr < narr; ++arr) {
        Real* s = arr == 0 ? sa : sb;
#pragma unroll 1
        for (int d = 0; d < DIM; ++d) {
            for (int t = lane; t < NL; t += 32) {
                Real l[NP], r[NP];
                vload_line<DIM, P>(s, t / NFP, d, t % NFP, l);
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    r[i] = Real(0);
#pragma unroll
                    for (int k = 0; k < NP; ++k) r[i] += pq[i][k] * l[k];
                }
                vstore_line<DIM, P>(s, t / NFP, d, t % NFP, r);
            }
            __syncwarp();
        }
    }
    Real* ae = a + e * NV * NSP;
    for (int k = lane; k < NV * NSP; k += 32) ae[k] = sa[VL::pt(k / NSP, k % NSP)];
    if (b) {
        Real* be = b + e * NV * NSP;
        for (int k = lane; k < NV * NSP; k += 32) be[k] = sb[VL::pt(k / NSP, k % NSP)];
    }
    if (uf_out) warp_write_traces<DIM, P, 32>(sa, uf_out + e * NF * NV * NFP, op, lane);
}

// Adaptive time step (Section 3.1: adaptive time stepping): per element
// lambda_e = max_sp (|V| + c) (p+1)^2 / h_e + max_sp (mu / rho) (p+1)^4 / h_e^2
// in double, h_e the element length (min over points and directions of
// 2 |J| / |S[d,:]|, precomputed); the candidate's maximum is kept by an
// atomic maximum on the bits of the non-negative double (order-independent).
template <int DIM, int P, typename Real>
__global__ void k_cfl(const Real* __restrict__ u, const Real* __restrict__ hlen, int64_t E,
                      const int64_t* __restrict__ cand_off, int ncand, const __grid_constant__ Phys<Real> ph,
                      unsigned long long* __restrict__ lam) {
    using Z = Sz<DIM, P>;
    constexpr int NSP = Z::NSP, NV = Z::NV;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t e = int64_t(blockIdx.x) * (blockDim.x >> 5) + warp;
    if (e >= E) return;
    const Real* ue = u + e * NV * NSP;
    double vmax = 0.0, numax = 0.0;
    for (int sp = lane; sp < NSP; sp += 32) {
        const double rho = double(ue[sp]);
        double m2 = 0.0;
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            const double m = double(ue[(1 + i) * NSP + sp]);
            m2 += m * m;
        }
        const double p = double(ph.gm1) * (double(ue[(NV - 1) * NSP + sp]) - 0.5 * m2 / rho);
        const double v = sqrt(m2) / rho + sqrt(double(ph.gamma) * p / rho);
        vmax = fmax(vmax, v);
        numax = fmax(numax, double(ph.mu) / rho);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        numax = fmax(numax, __shfl_xor_sync(0xffffffffu, numax, o));
    }
    if (lane == 0) {
        int c = 0;
        while (c + 1 < ncand && e >= cand_off[c + 1]) ++c;
        const double h = double(hlen[e]);
        const double k = double((P + 1) * (P + 1));
        double l = vmax * k / h;
        if (ph.viscous) l += numax * k * k / (h * h);
        atomicMax(lam + c, static_cast<unsigned long long>(__double_as_longlong(l)));
    }
}

// Wall force (Section 3.2): FORCE_BLOCKS blocks per candidate each sum, over
// a slice of that candidate's wall face points, w_fp (p N - tau.N) with N the
// element's outward area-weighted normal (into the body), p from the interior
// trace and tau.N the momentum entries of the wall's common viscous flux, in
// double, into part[c][block][DIM]; k_forces_fin adds the partial sums in a
// fixed order (deterministic) and updates fnow/fsum/fcnt in place
// (graph-replay safe).
template <int DIM, int P, typename Real>
__global__ void k_forces(const Real* __restrict__ uf, const Real* __restrict__ fvn,
                         const int32_t* __restrict__ wall_ef, const int64_t* __restrict__ wall_off,
                         const __grid_constant__ Ops<Real> op, const __grid_constant__ Geo<Real> g, Real gm1,
                         int viscous, double* __restrict__ part) {
    using Z = Sz<DIM, P>;
    constexpr int NP = Z::NP, NFP = Z::NFP, NF = Z::NF, NV = Z::NV;
    __shared__ double red[DIM][256];
    const int c = blockIdx.y;
    const int64_t b = wall_off[c], n = wall_off[c + 1] - b;
    double acc[DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i) acc[i] = 0.0;
    for (int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < n * NFP;
         w += int64_t(gridDim.x) * blockDim.x) {
        const int fp = int(w % NFP);
        const int32_t ef = wall_ef[b + w / NFP];
        const int64_t e = ef / NF;
        const int f = ef % NF;
        Real uL[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) uL[v] = uf[int64_t(ef) * NV * NFP + v * NFP + fp];
        const Real p = pressure<DIM>(uL, gm1);
        Real N[DIM];
        load_normal<DIM>(g, e, f, fp, N);
        double wt;
        if (DIM == 2) {
            wt = 0.0;
#pragma unroll
            for (int j = 0; j < NP; ++j) if (fp == j) wt = double(op.w[j]);
        } else {
            double wa = 0.0, wb = 0.0;
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                if (fp % NP == j) wa = double(op.w[j]);
                if (fp / NP == j) wb = double(op.w[j]);
            }
            wt = wa * wb;
        }
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            double fi = double(p) * double(N[i]);
            if (viscous) fi -= double(fvn[int64_t(ef) * NV * NFP + (1 + i) * NFP + fp]);
            acc[i] += wt * fi;
        }
    }
#pragma unroll
    for (int i = 0; i < DIM; ++i) red[i][threadIdx.x] = acc[i];
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
#pragma unroll
            for (int i = 0; i < DIM; ++i) red[i][threadIdx.x] += red[i][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int i = 0; i < DIM; ++i) part[(int64_t(c) * gridDim.x + blockIdx.x) * 3 + i] = red[i][0];
}

// one warp per candidate: lane l adds partial sums l, l+32, ..., then a fixed
// butterfly adds the lanes (the same order on every call)
static __global__ void k_forces_fin(const double* __restrict__ part, int nblk, double* __restrict__ fnow,
                                    double* __restrict__ fsum, double* __restrict__ fcnt) {
    const int c = blockIdx.x, lane = threadIdx.x & 31;
    double s[3] = {0.0, 0.0, 0.0};
    for (int k = lane; k < nblk; k += 32)
#pragma unroll
        for (int i = 0; i < 3; ++i) s[i] += part[(int64_t(c) * nblk + k) * 3 + i];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[i] += __shfl_xor_sync(0xffffffffu, s[i], o);
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            fnow[c * 3 + i] = s[i];
            fsum[c * 3 + i] += s[i];
        }
        fcnt[c] += 1.0;
    }
}

// FW-H data-surface sampling (Section 3.1): one warp per surface point
// evaluates the element's tensor Lagrange interpolant (1D weights pw
// [npts][DIM][NP] precomputed at the located reference coordinates) and
// stores (rho, V_1, V_2, V_3, p) minus the free stream into record *count.
// counter[0] = records written, counter[1] = steps seen, counter[2] = overflow;
// the kernel samples only on steps that are multiples of `every`.
template <int DIM, int P, typename Real>
__global__ void k_sample(const Real* __restrict__ u, const int64_t* __restrict__ pe,
                         const Real* __restrict__ pw, int npts, Phys<Real> ph, Real* __restrict__ hist,
                         const int* __restrict__ count, int cap, int every) {
    using Z = Sz<DIM, P>;
    constexpr int NP = Z::NP, NSP = Z::NSP, NV = Z::NV;
    const int lane = threadIdx.x & 31;
    const int k = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
    if (k >= npts) return;
    if (count[1] % every != 0) return;
    const int rec = count[0];
    if (rec >= cap) return;
    const Real* ue = u + pe[k] * NV * NSP;
    const Real* wk = pw + int64_t(k) * DIM * NP;
    Real acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = Real(0);
    for (int sp = lane; sp < NSP; sp += 32) {
        Real wt = wk[sp % NP];
        wt *= wk[NP + (sp / NP) % NP];
        if (DIM == 3) wt *= wk[2 * NP + sp / (NP * NP)];
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += wt * ue[v * NSP + sp];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], o);
    if (lane == 0) {
        const Real rho = acc[0];
        const Real p = pressure<DIM>(acc, ph.gm1);
        Real* dst = hist + (int64_t(rec) * npts + k) * 5;
        dst[0] = rho - ph.rho_inf;
#pragma unroll
        for (int i = 0; i < 3; ++i) dst[1 + i] = (i < DIM) ? acc[1 + i] / rho - ph.vel_inf[i] : Real(0);
        dst[4] = p - ph.p_inf;
    }
}

// advances the counters after the sampling kernel of the same step
static __global__ void k_bump(int* count, int cap, int every) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (count[1] % every == 0) {
            if (count[0] < cap) count[0] += 1;
            else count[2] = 1;
        }
        count[1] += 1;
    }
}

// Volume integrals (double) of the conserved variables and of the kinetic
// energy over elements [e_first, e_first + ne): one partial row per block.
template <int DIM, int P, typename Real>
__global__ void k_integrals(const Real* __restrict__ u, int64_t e_first, int64_t ne,
                            const __grid_constant__ Ops<Real> op, const __grid_constant__ Geo<Real> g,
                            double* __restrict__ partial) {
    using Z = Sz<DIM, P>;
    constexpr int NP = Z::NP, NSP = Z::NSP, NV = Z::NV;
    __shared__ double red[NV + 1][256];
    // each thread sums its points in the working precision, blocks in double
    Real acc[NV + 1];
#pragma unroll
    for (int v = 0; v <= NV; ++v) acc[v] = Real(0);
    for (int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < ne * NSP;
         w += int64_t(gridDim.x) * blockDim.x) {
        const int64_t e = e_first + w / NSP;
        const int sp = int(w % NSP);
        Real w0 = Real(0), w1 = Real(0), w2 = Real(1);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            if (sp % NP == j) w0 = op.w[j];
            if ((sp / NP) % NP == j) w1 = op.w[j];
            if (DIM == 3 && sp / (NP * NP) == j) w2 = op.w[j];
        }
        const Real wt = w0 * w1 * w2 * g.J[e * g.sJ_e + sp * g.sJ_sp];  // integrals use |J| itself
        const Real* ue = u + e * NV * NSP + sp;
        Real m2 = Real(0);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const Real x = ue[v * NSP];
            acc[v] += wt * x;
            if (v >= 1 && v <= DIM) m2 += x * x;
        }
        acc[NV] += wt * Real(0.5) * m2 / ue[0];
    }
#pragma unroll
    for (int v = 0; v <= NV; ++v) red[v][threadIdx.x] = double(acc[v]);
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
#pragma unroll
            for (int v = 0; v <= NV; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int v = 0; v <= NV; ++v) partial[blockIdx.x * (NV + 1) + v] = red[v][0];
}

}  // namespace frk
