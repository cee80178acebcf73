// Kernels of the elements of reduced degree Q < P inside a degree-P mesh (the
// variable solution degree of Section 3.1, P0 far from the body up to P3 or
// P4 near it).  Such an element is a degree-Q FR element on its own
// (Q+1)^DIM GL points whose faces keep the degree-P flux points of the mesh:
// its state is stored as the values of its degree-Q polynomial at the
// degree-P points (so traces, sampling and state transfers are those of a
// degree-P element), the face data at the degree-P face points reach it
// through the L2 projection onto degree Q along each face direction (a
// mortar), and its residual, evaluated at its Q points with degree-Q
// operators, goes back to the degree-P points as the polynomial it is.
//
// One warp per element, one element per block; every array in shared memory
// in the canonical layout (point i0 + N i1 + N^2 i2, face point a + N b with a
// the lower of the face's two directions), the operator matrices copied to
// shared memory first (their indices vary across lanes).
#pragma once

#include "fr_kernels.cuh"

namespace frk {

// shared copy of the degree-Q operators of Red (row stride MAXNP)
template <typename Real>
struct RedOps {
    Real Iqp[MAXNP * MAXNP], Ipq[MAXNP * MAXNP], Pqp[MAXNP * MAXNP], D[MAXNP * MAXNP];
    Real lm[MAXNP], lp[MAXNP], hm[MAXNP], hp[MAXNP];
    Real plm[MAXNP], plp[MAXNP];   // degree-P line ends (traces)
};

template <typename Real>
__device__ __forceinline__ void red_load_ops(RedOps<Real>* so, const Red<Real>& rd, const Ops<Real>& op, int lane) {
    for (int k = lane; k < MAXNP * MAXNP; k += 32) {
        so->Iqp[k] = rd.Iqp[k];
        so->Ipq[k] = rd.Ipq[k];
        so->Pqp[k] = rd.Pqp[k];
        so->D[k] = rd.D[k];
    }
    if (lane < MAXNP) {
        so->lm[lane] = rd.lm[lane];
        so->lp[lane] = rd.lp[lane];
        so->hm[lane] = rd.hm[lane];
        so->hp[lane] = rd.hp[lane];
        so->plm[lane] = op.lm[lane];
        so->plp[lane] = op.lp[lane];
    }
}

// f(t) for t = lane, lane + 32, ... < TOT, unrolled so that the loads of the
// iterations are issued together
template <int TOT, typename Fn>
__device__ __forceinline__ void lanes(int lane, Fn&& f) {
#pragma unroll
    for (int it = 0; it < (TOT + 31) / 32; ++it) {
        const int t = lane + 32 * it;
        if (TOT % 32 == 0 || t < TOT) f(t);
    }
}

// out[v][..] = sum_j M[o][j] in[v][.. j ..] along direction D of a tensor
// [NV][N2][N1][N0] (direction 0 fastest); the output has extent MO along D
template <int NV, int N0, int N1, int N2, int D, int MO, typename Real>
__device__ __forceinline__ void tapply(const Real* in, Real* out, const Real* M, int lane) {
    constexpr int O0 = D == 0 ? MO : N0, O1 = D == 1 ? MO : N1, O2 = D == 2 ? MO : N2;
    constexpr int NI = D == 0 ? N0 : D == 1 ? N1 : N2;
    constexpr int ST = D == 0 ? 1 : D == 1 ? N0 : N0 * N1;
    lanes<NV * O0 * O1 * O2>(lane, [&](int t) {
        int r = t;
        const int i0 = r % O0;
        r /= O0;
        const int i1 = r % O1;
        r /= O1;
        const int i2 = r % O2;
        const int v = r / O2;
        const int od = D == 0 ? i0 : D == 1 ? i1 : i2;
        const int b0 = D == 0 ? 0 : i0, b1 = D == 1 ? 0 : i1, b2 = D == 2 ? 0 : i2;
        const Real* src = in + ((v * N2 + b2) * N1 + b1) * N0 + b0;
        Real acc = Real(0);
#pragma unroll
        for (int j = 0; j < NI; ++j) acc += M[od * MAXNP + j] * src[j * ST];
        out[t] = acc;
    });
}

// M [NO][NI] along every direction of volume data [NV][NI^DIM] -> [NV][NO^DIM]
// (t1, t2: scratch of NV * max(NI, NO)^(DIM-1) * min(NI, NO) values each)
template <int DIM, int NV, int NI, int NO, typename Real>
__device__ __forceinline__ void vol_apply(const Real* in, Real* t1, Real* t2, Real* out, const Real* M, int lane) {
    if constexpr (DIM == 2) {
        tapply<NV, NI, NI, 1, 0, NO>(in, t1, M, lane);
        __syncwarp();
        tapply<NV, NO, NI, 1, 1, NO>(t1, out, M, lane);
    } else {
        tapply<NV, NI, NI, NI, 0, NO>(in, t1, M, lane);
        __syncwarp();
        tapply<NV, NO, NI, NI, 1, NO>(t1, t2, M, lane);
        __syncwarp();
        tapply<NV, NO, NO, NI, 2, NO>(t2, out, M, lane);
    }
    __syncwarp();
}

// M [NO][NI] along the DIM - 1 directions of face data [NV][NI^(DIM-1)] (t:
// scratch of NV * NI * NO values in 3D)
template <int DIM, int NV, int NI, int NO, typename Real>
__device__ __forceinline__ void face_apply(const Real* in, Real* t, Real* out, const Real* M, int lane) {
    if constexpr (DIM == 2) {
        tapply<NV, NI, 1, 1, 0, NO>(in, out, M, lane);
    } else {
        tapply<NV, NI, NI, 1, 0, NO>(in, t, M, lane);
        __syncwarp();
        tapply<NV, NO, NI, 1, 1, NO>(t, out, M, lane);
    }
    __syncwarp();
}

// shared-memory plan of one reduced element (Real units; every part keeps
// double data 8-byte aligned)
constexpr int red_ev(int n) { return (n + 1) & ~1; }
constexpr int red_max(int a, int b) { return a > b ? a : b; }

template <int DIM, int P, int Q>
struct RedSz {
    using ZP = Sz<DIM, P>;
    static constexpr int NQ = Q + 1;
    static constexpr int NSQ = DIM == 2 ? NQ * NQ : NQ * NQ * NQ;
    static constexpr int NFQ = DIM == 2 ? NQ : NQ * NQ;
    static constexpr int NV = ZP::NV, NP = ZP::NP, NSP = ZP::NSP, NFP = ZP::NFP, NF = ZP::NF;
    static constexpr int NG = DIM * DIM * NSQ + NSQ;          // metric terms and 1/|J| at the Q points
    // scratch of the volume passes (two halves) and of the face projections
    static constexpr int NT = red_ev(NV * (DIM == 2 ? NP * NQ : NP * NP * NQ));
    static constexpr int NSCR = red_max(2 * NT, red_ev(2 * NF * NV * NP * NQ));
    // residual kernel: state, metrics, u_q (then R_q), the jumps and common
    // fluxes at the P face points (then F~_d, then R at the P points), their
    // projections, scratch
    static constexpr int su = 0;
    static constexpr int geo = su + red_ev(NV * NSP);
    static constexpr int uq = geo + red_ev(NG);
    static constexpr int fa = uq + red_ev(NV * NSQ);
    static constexpr int nfa = red_max(2 * NF * NV * NFP, red_max(red_ev(DIM * NV * NSQ), red_ev(NV * NSP)));
    static constexpr int fq = fa + red_ev(nfa);                   // [2][NF][NV][NFQ]
    static constexpr int scr = fq + red_ev(2 * NF * NV * NFQ);
    static constexpr int total = scr + NSCR;
    // face kernel: state, metrics, u_q, the jumps at the P face points, their
    // projections, the uncorrected gradient, every face's G at the Q face
    // points, scratch
    static constexpr int f_su = 0;
    static constexpr int f_geo = f_su + red_ev(NV * NSP);
    static constexpr int f_uq = f_geo + red_ev(NG);
    static constexpr int f_sj = f_uq + red_ev(NV * NSQ);
    static constexpr int f_jq = f_sj + red_ev(NF * NV * NFP);
    static constexpr int f_gd = f_jq + red_ev(NF * NV * NFQ);
    static constexpr int f_gq = f_gd + red_ev(NV * DIM * NSQ);
    static constexpr int f_scr = f_gq + red_ev(NF * NV * DIM * NFQ);
    static constexpr int f_total = f_scr + NSCR;
};

// per-element time step, RK4 or coefficient-form stage update of one value
// (the arithmetic of k_residual's epilogue)
template <typename Real>
__device__ __forceinline__ Real red_stage(const Stage<Real>& st, Real dt, Real r, Real u, Real pu0, Real pacc,
                                          int64_t gi, bool& bad) {
    Real u0v = Real(0), accv = Real(0);
    if (st.stage >= 2) {
        u0v = pu0;
        accv = pacc;
    }
    if (st.ls) {
        const Real fdt = st.cf * dt, cdt = st.cc * dt;
        if (st.stage == 1) u0v = u;
        const Real an = st.stage == 1 ? mul_rn(fdt, r) : fma_rn(fdt, r, mul_rn(st.ce, accv));
        Real nu = fma_rn(st.cd, an, mul_rn(st.ca, u0v));
        nu = fma_rn(cdt, r, fma_rn(st.cb, u, nu));
        if (st.last) {
            st.u0[gi] = nu;
            bad = bad || not_finite(nu);
        } else {
            st.acc[gi] = an;
            st.us[gi] = nu;
        }
        return nu;
    }
    switch (st.stage) {
        case 0:
            st.R[gi] = r;
            return u;
        case 1: {
            st.acc[gi] = mul_rn(dt * Real(1.0 / 6.0), r);
            const Real nu = fma_rn(dt * Real(0.5), r, u);
            st.us[gi] = nu;
            return nu;
        }
        case 2: {
            st.acc[gi] = fma_rn(dt * Real(1.0 / 3.0), r, accv);
            const Real nu = fma_rn(dt * Real(0.5), r, u0v);
            st.us[gi] = nu;
            return nu;
        }
        case 3: {
            st.acc[gi] = fma_rn(dt * Real(1.0 / 3.0), r, accv);
            const Real nu = fma_rn(dt, r, u0v);
            st.us[gi] = nu;
            return nu;
        }
        default: {
            const Real nu = fma_rn(dt * Real(1.0 / 6.0), r, add_rn(u0v, accv));
            st.u0[gi] = nu;
            bad = bad || not_finite(nu);
            return nu;
        }
    }
}

// The degree-P face points of one element: trace u_L, outside state, jump
// u_c - u_L into sj[f][v][fp]; with FC also the common normal flux (Rusanov
// minus the common viscous flux) into sc[f][v][fp].
template <int DIM, int P, typename Real, bool FC, bool VISC>
__device__ __forceinline__ void red_face_points(int64_t e, const int (&codes)[2 * DIM], const Real* __restrict__ uf,
                                                const Real* __restrict__ fvn, const Phys<Real>& ph,
                                                const Geo<Real>& g, Real* sj, Real* sc, int lane) {
    using Z = Sz<DIM, P>;
    constexpr int NP = Z::NP, NFP = Z::NFP, NF = Z::NF, NV = Z::NV;
    lanes<NF * NFP>(lane, [&](int t) {
        const int f = t / NFP, fp = t % NFP;
        int code = codes[0];
#pragma unroll
        for (int k = 1; k < NF; ++k)
            if (f == k) code = codes[k];
        Real uL[NV], uR[NV], uc[NV], N[DIM];
        const Real* tf = uf + (e * NF + f) * NV * NFP + fp;
#pragma unroll
        for (int v = 0; v < NV; ++v) uL[v] = tf[v * NFP];
        load_normal<DIM>(g, e, f, fp, N);
        int fpn = 0;
        if (code >= 0) {
            fpn = omap<DIM, NP>(code & 7, fp);
            const Real* un = uf + int64_t(code >> 3) * NV * NFP + fpn;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                uR[v] = un[v * NFP];
                uc[v] = Real(0.5) * (uL[v] + uR[v]);
            }
        } else {
            bc_state<DIM>(-code, uL, N, ph, uR, uc);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) sj[(f * NV + v) * NFP + fp] = uc[v] - uL[v];
        if constexpr (FC) {
            Real Fc[NV];
            rusanov<DIM>(uL, uR, N, ph.gamma, ph.gm1, Fc);
            if constexpr (VISC) {
                const Real* own = fvn + (e * NF + f) * NV * NFP + fp;
                if (code >= 0) {
                    const Real* nb = fvn + int64_t(code >> 3) * NV * NFP + fpn;
#pragma unroll
                    for (int v = 0; v < NV; ++v) Fc[v] -= Real(0.5) * (own[v * NFP] - nb[v * NFP]);
                } else {
#pragma unroll
                    for (int v = 0; v < NV; ++v) Fc[v] -= own[v * NFP];
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) sc[(f * NV + v) * NFP + fp] = Fc[v];
        }
    });
}

// the neighbour codes of element e, in every lane
template <int NF, typename Real>
__device__ __forceinline__ void red_codes_of(const Geo<Real>& g, int64_t e, int (&codes)[NF], int lane) {
    const int mine = lane < NF ? g.nbr[e * NF + lane] : 0;
#pragma unroll
    for (int f = 0; f < NF; ++f) codes[f] = __shfl_sync(0xffffffffu, mine, f);
}

// state, metric terms and 1/|J| of reduced element k into shared memory
template <int DIM, int P, int Q, typename Real>
__device__ __forceinline__ void red_stage_in(const Red<Real>& rd, int k, int64_t e, const Real* __restrict__ u,
                                             Real* su, Real* geo, int lane) {
    using RS = RedSz<DIM, P, Q>;
    const Real* ue = u + e * RS::NV * RS::NSP;
    lanes<RS::NV * RS::NSP>(lane, [&](int t) { su[t] = ue[t]; });
    const Real* Sq = rd.S + int64_t(k) * rd.sS;
    const Real* iJq = rd.iJ + int64_t(k) * rd.sJ;
    lanes<RS::NG>(lane, [&](int t) { geo[t] = t < DIM * DIM * RS::NSQ ? Sq[t] : iJq[t - DIM * DIM * RS::NSQ]; });
}

// BR2 face gradients of the reduced elements of degree Q and their own viscous
// normal fluxes at the degree-P face points: G = I_f[grad_D u_q] +
// eta I_f[r_f] at the Q face points (r_f the degree-Q lifting of face f's
// projected jump alone), evaluated at the degree-P face points; fvn gets
// F_vis(u_f, G).N, or on a boundary face the common viscous flux
// F_vis(u_b, G).N (energy entry zero at an adiabatic wall).
template <int DIM, int P, int Q, typename Real>
__global__ void k_red_face(const __grid_constant__ Red<Real> rd, const Real* __restrict__ u,
                           const Real* __restrict__ uf, Real* __restrict__ fvn, const __grid_constant__ Ops<Real> op,
                           const __grid_constant__ Phys<Real> ph, const __grid_constant__ Geo<Real> g) {
    using RS = RedSz<DIM, P, Q>;
    constexpr int NV = RS::NV, NP = RS::NP, NFP = RS::NFP, NF = RS::NF;
    constexpr int NQ = RS::NQ, NSQ = RS::NSQ, NFQ = RS::NFQ;
    extern __shared__ __align__(16) unsigned char smem[];
    RedOps<Real>* so = reinterpret_cast<RedOps<Real>*>(smem);
    Real* base = reinterpret_cast<Real*>(smem + ((sizeof(RedOps<Real>) + 15) & ~size_t(15)));
    Real* su = base + RS::f_su;
    Real* geo = base + RS::f_geo;   // S [DIM*DIM][NSQ], 1/|J| [NSQ]
    Real* uq = base + RS::f_uq;
    Real* sj = base + RS::f_sj;     // jumps at the degree-P face points [NF][NV][NFP]
    Real* jq = base + RS::f_jq;     // projected jumps [NF][NV][NFQ]
    Real* gD = base + RS::f_gd;     // uncorrected gradient [NV][DIM][NSQ]
    Real* gq = base + RS::f_gq;     // G at the Q face points [NF][NV][DIM][NFQ]
    Real* scr = base + RS::f_scr;
    const int lane = threadIdx.x;
    const int k = blockIdx.x;
    if (k >= rd.n) return;
    const int64_t e = rd.elem[k];
    red_load_ops(so, rd, op, lane);
    int codes[NF];
    red_codes_of<NF>(g, e, codes, lane);
    red_stage_in<DIM, P, Q>(rd, k, e, u, su, geo, lane);
    red_face_points<DIM, P, Real, false, true>(e, codes, uf, nullptr, ph, g, sj, nullptr, lane);
    __syncwarp();
    vol_apply<DIM, NV, NP, NQ>(su, scr, scr + RS::NT, uq, so->Iqp, lane);
    face_apply<DIM, NF * NV, NP, NQ>(sj, scr, jq, so->Pqp, lane);
    const Real* iJq = geo + DIM * DIM * NSQ;
    // uncorrected physical gradient at the Q points
    lanes<NV * NSQ>(lane, [&](int t) {
        const int v = t / NSQ, pt = t % NSQ;
        Real qd[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            int fpq, jl;
            sp_split<DIM, NQ>(pt, d, fpq, jl);
            Real a = Real(0);
#pragma unroll
            for (int j = 0; j < NQ; ++j) a += so->D[jl * MAXNP + j] * uq[v * NSQ + line_sp<DIM, NQ>(d, fpq, j)];
            qd[d] = a;
        }
        const Real iJ = iJq[pt];
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
            Real a = Real(0);
#pragma unroll
            for (int d = 0; d < DIM; ++d) a += geo[(d * DIM + i) * NSQ + pt] * qd[d];
            gD[(v * DIM + i) * NSQ + pt] = a * iJ;
        }
    });
    __syncwarp();
    // every face's G at its Q face points
    lanes<NF * NV * DIM * NFQ>(lane, [&](int t) {
        const int fq = t % NFQ, r = t / NFQ, i = r % DIM, v = (r / DIM) % NV, f = r / (DIM * NV);
        const int d = f >> 1, s = f & 1;
        const Real* lv = s ? so->lp : so->lm;
        const Real* hv = s ? so->hp : so->hm;
        const Real nsg = s ? Real(1) : Real(-1);
        Real a = Real(0), lc = Real(0);
#pragma unroll
        for (int j = 0; j < NQ; ++j) {
            const int pt = line_sp<DIM, NQ>(d, fq, j);
            a += lv[j] * gD[(v * DIM + i) * NSQ + pt];
            lc += lv[j] * (nsg * (geo[(d * DIM + i) * NSQ + pt] * iJq[pt]) * hv[j]);
        }
        gq[t] = a + ph.eta * (lc * jq[(f * NV + v) * NFQ + fq]);
    });
    __syncwarp();
    // at each degree-P face point: G evaluated there (the degree-Q face
    // polynomial at the P point), the viscous normal flux
    lanes<NF * NFP>(lane, [&](int t) {
        const int f = t / NFP, fp = t % NFP;
        int code = codes[0];
#pragma unroll
        for (int kk = 1; kk < NF; ++kk)
            if (f == kk) code = codes[kk];
        Real wa[NQ], wb[DIM == 3 ? NQ : 1];
        const int ap = DIM == 3 ? fp % NP : fp, bp = DIM == 3 ? fp / NP : 0;
#pragma unroll
        for (int j = 0; j < NQ; ++j) wa[j] = so->Ipq[ap * MAXNP + j];
        if constexpr (DIM == 3) {
#pragma unroll
            for (int j = 0; j < NQ; ++j) wb[j] = so->Ipq[bp * MAXNP + j];
        } else {
            wb[0] = Real(1);
        }
        Real G[NV][DIM];
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int i = 0; i < DIM; ++i) {
                const Real* gv = gq + ((f * NV + v) * DIM + i) * NFQ;
                Real a = Real(0);
#pragma unroll
                for (int jb = 0; jb < (DIM == 3 ? NQ : 1); ++jb) {
                    Real r = Real(0);
#pragma unroll
                    for (int ja = 0; ja < NQ; ++ja) r += wa[ja] * gv[jb * NQ + ja];
                    a += wb[jb] * r;
                }
                G[v][i] = a;
            }
        Real uL[NV], N[DIM], Fn[NV];
        const Real* tf = uf + (e * NF + f) * NV * NFP + fp;
#pragma unroll
        for (int v = 0; v < NV; ++v) uL[v] = tf[v * NFP];
        load_normal<DIM>(g, e, f, fp, N);
        if (code >= 0) {
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
    });
}

// Residual of the reduced elements of degree Q, the stage update at the
// degree-P points and the traces of the new stage state (the counterpart of
// k_residual): common fluxes and jumps at the degree-P face points, projected
// onto degree Q; degree-Q corrected gradient, flux, divergence and correction
// at the Q points; R_q = -div / |J|; R = I_pq R_q.
template <int DIM, int P, int Q, typename Real, bool VISC>
__global__ void k_red_resid(const __grid_constant__ Red<Real> rd, const Real* __restrict__ u,
                            const Real* __restrict__ uf, const Real* __restrict__ fvn,
                            const __grid_constant__ Ops<Real> op, const __grid_constant__ Phys<Real> ph,
                            const __grid_constant__ Geo<Real> g, const __grid_constant__ Stage<Real> st) {
    using RS = RedSz<DIM, P, Q>;
    constexpr int NV = RS::NV, NP = RS::NP, NSP = RS::NSP, NFP = RS::NFP, NF = RS::NF;
    constexpr int NQ = RS::NQ, NSQ = RS::NSQ, NFQ = RS::NFQ;
    extern __shared__ __align__(16) unsigned char smem[];
    RedOps<Real>* so = reinterpret_cast<RedOps<Real>*>(smem);
    Real* base = reinterpret_cast<Real*>(smem + ((sizeof(RedOps<Real>) + 15) & ~size_t(15)));
    Real* su = base + RS::su;
    Real* geo = base + RS::geo;                  // S [DIM*DIM][NSQ], 1/|J| [NSQ]
    Real* uq = base + RS::uq;
    Real* sj = base + RS::fa;                    // jumps [NF][NV][NFP], then
    Real* sc = sj + NF * NV * NFP;               // common normal fluxes [NF][NV][NFP]
    Real* Ft = base + RS::fa;                    // then F~_d [DIM][NV][NSQ]
    Real* jq = base + RS::fq;                    // projected jumps [NF][NV][NFQ], then
    Real* fq = jq + NF * NV * NFQ;               // projected fluxes [NF][NV][NFQ]
    Real* scr = base + RS::scr;
    const int lane = threadIdx.x;
    const int k = blockIdx.x;
    if (k >= rd.n) return;
    const int64_t e = rd.elem[k];
    red_load_ops(so, rd, op, lane);
    int codes[NF];
    red_codes_of<NF>(g, e, codes, lane);
    red_stage_in<DIM, P, Q>(rd, k, e, u, su, geo, lane);
    // the stage arrays (needed at the end): issue their loads now
    constexpr int NSW = (NV * NSP + 31) / 32;
    Real pu0[NSW], pacc[NSW];
    if (st.stage >= 2) {
#pragma unroll
        for (int it = 0; it < NSW; ++it) {
            const int t = lane + 32 * it;
            if (t < NV * NSP) {
                pu0[it] = st.u0[e * NV * NSP + t];
                pacc[it] = st.acc[e * NV * NSP + t];
            }
        }
    }
    red_face_points<DIM, P, Real, true, VISC>(e, codes, uf, fvn, ph, g, sj, sc, lane);
    __syncwarp();
    vol_apply<DIM, NV, NP, NQ>(su, scr, scr + RS::NT, uq, so->Iqp, lane);
    face_apply<DIM, 2 * NF * NV, NP, NQ>(sj, scr, jq, so->Pqp, lane);   // jumps and fluxes at once
    const Real* iJq = geo + DIM * DIM * NSQ;
    // flux at the Q points: F~_d = sum_i S[d][i] (F_inv - F_vis)_i
    lanes<NSQ>(lane, [&](int pt) {
        Real S[DIM * DIM], uu[NV], F[NV][DIM];
#pragma unroll
        for (int kk = 0; kk < DIM * DIM; ++kk) S[kk] = geo[kk * NSQ + pt];
#pragma unroll
        for (int v = 0; v < NV; ++v) uu[v] = uq[v * NSQ + pt];
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
            const Real iJ = iJq[pt];
            Real G[NV][DIM];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                Real qd[DIM];
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    int fpq, jl;
                    sp_split<DIM, NQ>(pt, d, fpq, jl);
                    Real a = Real(0);
#pragma unroll
                    for (int j = 0; j < NQ; ++j)
                        a += so->D[jl * MAXNP + j] * uq[v * NSQ + line_sp<DIM, NQ>(d, fpq, j)];
                    a += so->hp[jl] * jq[((2 * d + 1) * NV + v) * NFQ + fpq] -
                         so->hm[jl] * jq[((2 * d) * NV + v) * NFQ + fpq];
                    qd[d] = a;
                }
#pragma unroll
                for (int i = 0; i < DIM; ++i) {
                    Real a = Real(0);
#pragma unroll
                    for (int d = 0; d < DIM; ++d) a += S[d * DIM + i] * qd[d];
                    G[v][i] = a * iJ;
                }
            }
            Real Fv[NV][DIM];
            visc_flux<DIM>(uu, G, ph.mu, ph.kappa, Fv);
#pragma unroll
            for (int v = 0; v < NV; ++v)
#pragma unroll
                for (int i = 0; i < DIM; ++i) F[v][i] -= Fv[v][i];
        }
        // (F~ lands in the face region, whose data are already projected; it
        // does not overlap u_q)
#pragma unroll
        for (int d = 0; d < DIM; ++d)
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                Real a = Real(0);
#pragma unroll
                for (int i = 0; i < DIM; ++i) a += S[d * DIM + i] * F[v][i];
                Ft[(d * NV + v) * NSQ + pt] = a;
            }
    });
    __syncwarp();
    // divergence plus correction, R_q = -div / |J| into u_q
    lanes<NV * NSQ>(lane, [&](int t) {
        const int v = t / NSQ, pt = t % NSQ;
        Real div = Real(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            int fpq, jl;
            sp_split<DIM, NQ>(pt, d, fpq, jl);
            const Real* Fd = Ft + (d * NV + v) * NSQ;
            Real a = Real(0), em = Real(0), ep = Real(0);
#pragma unroll
            for (int j = 0; j < NQ; ++j) {
                const Real x = Fd[line_sp<DIM, NQ>(d, fpq, j)];
                a += so->D[jl * MAXNP + j] * x;
                em += so->lm[j] * x;
                ep += so->lp[j] * x;
            }
            const Real cm = fq[((2 * d) * NV + v) * NFQ + fpq] + em;   // Fc.N - (-1) I_-[F~_d]
            const Real cp = fq[((2 * d + 1) * NV + v) * NFQ + fpq] - ep;
            div += a + so->hm[jl] * cm + so->hp[jl] * cp;
        }
        uq[t] = -div * iJq[pt];
    });
    __syncwarp();
    // R at the degree-P points (into the face region), the stage update, the
    // new state into su
    Real* Rp = base + RS::fa;
    vol_apply<DIM, NV, NQ, NP>(uq, scr, scr + RS::NT, Rp, so->Ipq, lane);
    const Real dt = st.dte ? st.dte[e] : st.dt;
    bool bad = false;
#pragma unroll
    for (int it = 0; it < NSW; ++it) {
        const int t = lane + 32 * it;
        if (t < NV * NSP) {
            const int64_t gi = e * NV * NSP + t;
            su[t] = red_stage(st, dt, Rp[t], su[t], pu0[it], pacc[it], gi, bad);
        }
    }
    if (st.nonfinite && __any_sync(0xffffffffu, bad) && lane == 0) {
        int c = 0;
        while (c + 1 < st.ncand && e >= st.cand_off[c + 1]) ++c;
        atomicOr(st.nonfinite + c, 1);
    }
    if (st.uf_next) {
        __syncwarp();
        Real* ufe = st.uf_next + e * NF * NV * NFP;
        lanes<NF * NV * NFP>(lane, [&](int t) {
            const int fp = t % NFP, fv = t / NFP, v = fv % NV, f = fv / NV;
            const int d = f >> 1;
            const Real* lv = (f & 1) ? so->plp : so->plm;
            Real a = Real(0);
#pragma unroll
            for (int j = 0; j < NP; ++j) a += lv[j] * su[v * NSP + line_sp<DIM, NP>(d, fp, j)];
            ufe[t] = a;
        });
    }
}

// dynamic shared memory of k_red_resid (face = false) and k_red_face
template <int DIM, int P, int Q, typename Real>
constexpr size_t smem_red(bool face) {
    return ((sizeof(RedOps<Real>) + 15) & ~size_t(15)) +
           size_t(face ? RedSz<DIM, P, Q>::f_total : RedSz<DIM, P, Q>::total) * sizeof(Real);
}

}  // namespace frk
