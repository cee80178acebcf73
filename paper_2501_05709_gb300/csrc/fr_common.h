// Shared declarations of the libfr host code and kernels (not part of the
// public ABI).  Plain structs passed to kernels by value.
#pragma once

#include <cstddef>
#include <cstdint>

#include "fr.h"

namespace frk {

constexpr int MAXNP = 5;  // p <= 4
constexpr int FORCE_BLOCKS = 64;  // wall-force partial sums per candidate

// 1D reference operators of one order p and correction kind, Section 1 (FR):
// lm/lp extrapolate a line of solution points to the xi=-1/+1 end, D is the
// solution-point derivative matrix D[i*MAXNP+j] = l_j'(x_i), hm/hp are the
// correction-derivative profiles (-g_L'(x_i) and g_R'(x_i)), w the GL
// weights; lhm/lhp = sum_j lm_j hm_j and sum_j lp_j hp_j.
template <typename Real>
struct Ops {
    Real lm[MAXNP];
    Real lp[MAXNP];
    Real D[MAXNP * MAXNP];
    Real hm[MAXNP];
    Real hp[MAXNP];
    Real w[MAXNP];
    Real dlm[MAXNP];  // l_j'(-1), derivative of the basis at the left end
    Real lhm, lhp;
};

// Gas and flow constants (Section 2.1, Eqs. 5-7) and the free stream.
template <typename Real>
struct Phys {
    Real gamma, gm1, mu, kappa, eta;
    Real rho_inf, p_inf, vel_inf[3];
    int viscous;
};

// Geometry arrays with strides: an affine mesh stores one metric set per
// element (sp/fp strides 0), a curved mesh one per solution/flux point.
//   S[e*sS_e + k*sS_k + sp*sS_sp], k = d*DIM + i   : |J| dxi_d/dx_i
//   J[e*sJ_e + sp*sJ_sp]                            : |J|   (iJ: 1/|J|, same strides)
//   N[(e*NF + f)*sN_f + fp*sN_fp + i]               : outward area-weighted normal
//   nbr[e*NF + f] = (ne*NF + nf)*8 + orientation, or -tag on boundary faces
template <typename Real>
struct Geo {
    const Real* S;
    const Real* J;
    const Real* iJ;
    const Real* N;
    const int32_t* nbr;
    int64_t sS_e, sS_k, sS_sp;
    int64_t sJ_e, sJ_sp;
    int64_t sN_f, sN_fp;
    // 1: every element is affine with a diagonal S (axis-aligned boxes; the
    // off-diagonal entries are exact zeros), so S^T q and S F take one term
    int diag;
    // 1: some element face lies on a boundary (0: fully periodic mesh)
    int bnd;
    // per-element polynomial degree when some element has a reduced degree
    // (null: every element has the mesh's degree); the element kernels of the
    // mesh's degree skip the reduced ones, which the kernels of Red handle
    const signed char* order = nullptr;
};

// Stage control for the fused residual/update kernel.  Classic RK4 (ls = 0):
//   stage 0: write R only (fr_residual)
//   stage 1: input u0;  acc = dt/6 k1;        us = u0 + dt/2 k1
//   stage 2: input us;  acc += dt/3 k2;       us = u0 + dt/2 k2
//   stage 3: input us;  acc += dt/3 k3;       us = u0 + dt k3
//   stage 4: input us;  u0 = u0 + acc + dt/6 k4
// Coefficient form (ls = 1), stage i >= 1 with input v (u0 at stage 1, us
// after) and k = R(v):
//   acc <- e acc + f dt k          (acc taken as 0 at stage 1)
//   out  = a u0 + b v + c dt k + d acc, evaluated as ((a u0 + d acc) + b v) + (c dt) k
//   out -> us, or -> u0 at the last stage (acc is then not written)
// uf_next (stages >= 1): traces of the stage's output state, for the next stage.
// dte (optional): per-element time step overriding dt.
// nonfinite (optional): the last stage sets nonfinite[c] when candidate c's
// new state holds a NaN or an infinity (candidate offsets cand_off[0..ncand]).
template <typename Real>
struct Stage {
    int stage;
    Real dt;
    const Real* dte;
    Real* R;          // stage 0 output
    Real* u0;
    Real* us;
    Real* acc;
    Real* uf_next;
    int* nonfinite = nullptr;
    const int64_t* cand_off = nullptr;
    int ncand = 0;
    int ls = 0;       // 1: coefficient form
    int last = 0;     // coefficient form: this stage writes u0
    Real ca = 0, cb = 0, cc = 0, cd = 0, ce = 0, cf = 0;
};

// Bit test for NaN and infinity (exponent field all ones), independent of
// fast-math flags.
__host__ __device__ inline bool not_finite(float x) {
    union { float f; uint32_t u; } b;
    b.f = x;
    return (b.u & 0x7f800000u) == 0x7f800000u;
}
__host__ __device__ inline bool not_finite(double x) {
    union { double f; uint64_t u; } b;
    b.f = x;
    return (b.u & 0x7ff0000000000000ull) == 0x7ff0000000000000ull;
}

// Energy source of Appendix D, Eq. D.1,
//   s(x, t) = sum_m A_m exp(-k_m |x - x_m|^2) sin(2 pi f_m t),
// for the nentry elements that carry one: elem[j], cand[j] and weights
// w[j][m][sp] = exp(-k_m |x_sp - x_m|^2); A, f per candidate [cand][MAXSRC]
// (unused slots A = 0); stage time t = tnow[cand] + cfac * dt (cfac = 0, 1/2,
// 1/2, 1 for stages 1-4; 0 for stage 0).
constexpr int MAXSRC = 4;
template <typename Real>
struct Src {
    int nentry = 0;
    const int32_t* elem = nullptr;
    const int32_t* cand = nullptr;
    const Real* w = nullptr;
    const double* A = nullptr;
    const double* f = nullptr;
    const double* tnow = nullptr;
    double cfac = 0.0;
};

// One warp per element; epb elements (warps) per block.
struct Launch {
    int epb;          // elements (warps) per block
    int threads;      // 32 * epb
};

// Variable polynomial order (sponge zones): the n listed elements keep their
// solution in the tensor-product space of degree cap[j] < p; pm[q] holds the
// 1D L2 projection onto degree q on the GL points, pm[q][i*MAXNP + j].
template <typename Real>
struct Sponge {
    int n = 0;
    const int32_t* elem = nullptr;
    const int32_t* cap = nullptr;
    Real pm[MAXNP][MAXNP * MAXNP];
};

// Elements of reduced degree Q < P inside a degree-P mesh (variable solution
// degree, Section 3.1): the n listed elements elem[k], their metric terms at
// the Q points S[k*sS + (d*DIM + i)*NSQ + pt] and 1/|J| iJ[k*sJ + pt] (the
// degree-P interpolants of the element's metrics evaluated there), and the
// degree-Q operators (row-major, row stride MAXNP): Iqp [NQ][NP] the
// Lagrange basis of the P points at the Q points, Ipq [NP][NQ] the reverse,
// Pqp [NQ][NP] the L2 projection onto degree Q (values at the Q points), D
// the degree-Q derivative matrix, lm/lp and hm/hp as in Ops for degree Q.
template <typename Real>
struct Red {
    int n = 0;
    const int32_t* elem = nullptr;
    const Real* S = nullptr;
    const Real* iJ = nullptr;
    int64_t sS = 0, sJ = 0;
    Real Iqp[MAXNP * MAXNP], Ipq[MAXNP * MAXNP], Pqp[MAXNP * MAXNP], D[MAXNP * MAXNP];
    Real lm[MAXNP], lp[MAXNP], hm[MAXNP], hp[MAXNP];
};

}  // namespace frk

// Host-side launchers implemented per precision and dimension.
namespace frl {

// Each returns a cudaError_t value (0 on success).  `op` holds the 1D
// operators of the context's order and correction (passed to the kernels as
// __grid_constant__ parameters).
template <typename Real, int DIM>
int traces(int P, const Real* u, Real* uf, int64_t E, const frk::Ops<Real>& op,
           frk::Launch lc, void* stream);

template <typename Real, int DIM>
int visc_face(int P, const Real* u, const Real* uf, Real* fvn, int64_t E,
              const frk::Ops<Real>& op, const frk::Phys<Real>& ph, const frk::Geo<Real>& g,
              frk::Launch lc, void* stream);

template <typename Real, int DIM>
int residual(int P, const Real* u, const Real* uf, const Real* fvn, int64_t E,
             const frk::Ops<Real>& op, const frk::Phys<Real>& ph, const frk::Geo<Real>& g,
             const frk::Stage<Real>& st, frk::Launch lc, void* stream);

template <typename Real, int DIM>
int forces(int P, const Real* uf, const Real* fvn, const int32_t* wall_ef, const int64_t* wall_off,
           int ncand, const frk::Ops<Real>& op, const frk::Geo<Real>& g, Real gm1, int viscous,
           double* part, double* fnow, double* fsum, double* fcnt, void* stream);

// count: device int[3] = records, steps seen, overflow flag
template <typename Real, int DIM>
int sample(int P, const Real* u, const int64_t* pe, const Real* pw, int npts, const frk::Phys<Real>& ph,
           Real* hist, int* count, int cap, int every, void* stream);

template <typename Real, int DIM>
int integrals(int P, const Real* u, int64_t e_first, int64_t ne, const frk::Ops<Real>& op,
              const frk::Geo<Real>& g, double* partial, int nblocks, void* stream);

// project a (and b if not null) of the sponge elements; traces of the
// projected a into uf_out when not null
template <typename Real, int DIM>
int sponge(int P, const frk::Sponge<Real>& sp, Real* a, Real* b, Real* uf_out, const frk::Ops<Real>& op,
           void* stream);

// energy source share of one stage (Src above) for the source elements
template <typename Real, int DIM>
int source_stage(int P, const frk::Src<Real>& src, const frk::Stage<Real>& st, const frk::Ops<Real>& op,
                 void* stream);

// per-candidate maximum spectral rate of the adaptive time step (lam holds
// the bits of non-negative doubles, zeroed by the caller)
template <typename Real, int DIM>
int cfl(int P, const Real* u, const Real* hlen, int64_t E, const int64_t* cand_off, int ncand,
        const frk::Phys<Real>& ph, unsigned long long* lam, void* stream);

// residual of the tensor-core precision modes (3D, P = 3 or 4; opm 1: TF32,
// 2: BF16x3), float data
int residual_tc3(int P, int opm, const float* u, const float* uf, const float* fvn, int64_t E,
                 const frk::Ops<float>& op, const frk::Phys<float>& ph, const frk::Geo<float>& g,
                 const frk::Stage<float>& st, frk::Launch lc, void* stream);

// the reduced-degree elements of Red (degree Q < P): BR2 face gradients and
// own viscous normal fluxes (red_face, viscous meshes), and the residual with
// the stage update and next traces (red_resid)
template <typename Real, int DIM>
int red_face(int P, int Q, const frk::Red<Real>& rd, const Real* u, const Real* uf, Real* fvn,
             const frk::Ops<Real>& op, const frk::Phys<Real>& ph, const frk::Geo<Real>& g, void* stream);

template <typename Real, int DIM>
int red_resid(int P, int Q, const frk::Red<Real>& rd, const Real* u, const Real* uf, const Real* fvn,
              const frk::Ops<Real>& op, const frk::Phys<Real>& ph, const frk::Geo<Real>& g,
              const frk::Stage<Real>& st, void* stream);

// threads per element of the element kernels (32 or 64; at 64 an element
// group synchronises on a named barrier, so a block holds at most 15 groups)
template <typename Real, int DIM>
int threads_per_element(int P);

// dynamic shared memory of kernel 0 (traces), 1 (viscous faces), 2 (residual);
// curved meshes stage per-point metrics and need more
template <typename Real, int DIM>
size_t smem_bytes(int P, int kernel, int epb, bool curved);

}  // namespace frl
