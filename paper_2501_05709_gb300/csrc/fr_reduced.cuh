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
// One warp per element, red_w elements per block.  The element's state is
// staged into shared memory by cp.async at kernel start; the face data (own
// and neighbour traces and viscous fluxes, normals), the metric terms at the
// Q points and the RK stage arrays are read from global memory where they
// are used, which keeps shared memory near 8 KB per element (FP32, P = 3).
// Every operator is applied along lines: a lane takes one line (or one face
// array), holds its values in registers and forms all outputs of the line
// with operator indices that are compile-time after unrolling, so the
// operator entries come from the constant bank of the __grid_constant__
// parameters.  Volume arrays in shared memory use the canonical layout
// (point i0 + N i1 + N^2 i2); face rows (face point a + N b, a the lower of
// the face's two directions) are padded to an odd stride.
#pragma once

#include <type_traits>

#include "fr_kernels.cuh"

namespace frk {

// f(std::integral_constant<int, I>) for I = I0 .. N-1: loops whose index
// must be a compile-time constant (a template argument)
template <int I, int N, typename F>
__device__ __forceinline__ void red_for(F&& f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>());
        red_for<I + 1, N>(f);
    }
}

__host__ __device__ constexpr int red_al(int n) { return (n + 3) & ~3; }   // regions start 16-byte aligned (float)
__host__ __device__ constexpr int red_mx(int a, int b) { return a > b ? a : b; }

template <int DIM, int P, int Q>
struct RedSz {
    static constexpr int NP = P + 1, NQ = Q + 1;
    static constexpr int NV = DIM + 2, NF = 2 * DIM;
    static constexpr int NSP = DIM == 2 ? NP * NP : NP * NP * NP;
    static constexpr int NSQ = DIM == 2 ? NQ * NQ : NQ * NQ * NQ;
    static constexpr int NFP = DIM == 2 ? NP : NP * NP;
    static constexpr int NFQ = DIM == 2 ? NQ : NQ * NQ;
    static constexpr int FA = NF * NV * NFP;           // one array of face data at the P points
    static constexpr int RW = NFP | 1;                  // padded row of face data at the P points
    // volume passes P <-> Q: the two intermediates of one direction sweep
    static constexpr int NY1 = NV * (DIM == 2 ? NP : NP * NP) * NQ;   // P -> Q after one direction (3D: also Q -> P after two)
    static constexpr int NY2 = DIM == 2 ? 0 : NV * NP * NQ * NQ;     // P -> Q after two directions (Q -> P after one)
    static constexpr int YB = red_al(NY1);                            // offset of the second intermediate
    static constexpr int NYS = YB + NY2;
    // residual kernel: state | face rows (jumps, then common fluxes, at the P
    // face points; then the volume scratch, q_d and F~_d) | projected jumps
    // and fluxes | u_q (then R_q)
    static constexpr int NM = red_mx(red_mx(2 * NF * NV * RW, NYS), DIM * NV * NSQ);
    static constexpr int su = 0;
    static constexpr int sm = su + red_al(NV * NSP);
    static constexpr int sjf = sm + red_al(NM);
    static constexpr int suq = sjf + red_al(2 * NF * NV * NFQ);
    static constexpr int total = suq + red_al(NV * NSQ);
    // face kernel: state | jump rows at the P face points (then the volume
    // scratch, q_d and the physical gradient) | projected jumps | u_q | G at
    // the Q face points of the two faces of one direction | G at their P face
    // points
    static constexpr int NM1 = red_mx(red_mx(NF * NV * RW, NYS), DIM * NV * NSQ);
    static constexpr int f_su = 0;
    static constexpr int f_sm = f_su + red_al(NV * NSP);
    static constexpr int f_jq = f_sm + red_al(NM1);
    static constexpr int f_uq = f_jq + red_al(NF * NV * NFQ);
    static constexpr int f_gq = f_uq + red_al(NV * NSQ);
    static constexpr int f_gp = f_gq + red_al(2 * NV * DIM * NFQ);
    static constexpr int f_total = f_gp + red_al(2 * NV * DIM * RW);
};

// elements (warps) per block: 4 when their shared memory allows
template <int DIM, int P, int Q, typename Real>
__host__ __device__ constexpr int red_w(bool face) {
    const size_t per = size_t(face ? RedSz<DIM, P, Q>::f_total : RedSz<DIM, P, Q>::total) * sizeof(Real);
    return per * 4 <= 200 * 1024 ? 4 : per * 2 <= 200 * 1024 ? 2 : 1;
}

// dynamic shared memory of one block of k_red_resid (face = false) or k_red_face
template <int DIM, int P, int Q, typename Real>
__host__ __device__ constexpr size_t smem_red(bool face) {
    return size_t(red_w<DIM, P, Q, Real>(face)) *
           size_t(face ? RedSz<DIM, P, Q>::f_total : RedSz<DIM, P, Q>::total) * sizeof(Real);
}

// Lines along direction D of NB batches of a tensor with extents (A0, A1, A2)
// (A0 fastest; A2 = 1 in 2D): task t (one line) -> batch b and line index r
// over the two other directions (lower first), which for a cube is the face
// point of the line; in/out offsets of the line's first point and strides.
template <int A0, int A1, int A2, int D, int MO>
struct LineMap {
    static constexpr int NI = D == 0 ? A0 : D == 1 ? A1 : A2;     // input points per line
    static constexpr int E0 = D == 0 ? A1 : A0;                   // the other two extents
    static constexpr int E1 = D == 2 ? A1 : A2;
    static constexpr int NL = E0 * E1;                            // lines per batch
    static constexpr int V = A0 * A1 * A2;                        // input batch size
    static constexpr int VO = V / NI * MO;                        // output batch size
    static constexpr int IS = D == 0 ? 1 : D == 1 ? A0 : A0 * A1;  // input stride along D
    static constexpr int OS = D == 0 ? 1 : D == 1 ? A0 : A0 * A1;  // output stride along D
    __device__ __forceinline__ static int ib(int b, int r) {
        if constexpr (D == 0) return b * V + A0 * r;
        else if constexpr (D == 1) return b * V + r % A0 + A0 * A1 * (r / A0);
        else return b * V + r;
    }
    __device__ __forceinline__ static int ob(int b, int r) {
        if constexpr (D == 0) return b * VO + MO * r;
        else if constexpr (D == 1) return b * VO + r % A0 + A0 * MO * (r / A0);
        else return b * VO + r;
    }
};

// load the NI values of a line (a 16-byte vector when the line is one float4)
template <int NI, int IS, typename Real>
__device__ __forceinline__ void red_ld(const Real* p, Real (&x)[NI]) {
    if constexpr (NI == 4 && IS == 1 && sizeof(Real) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        x[0] = q.x; x[1] = q.y; x[2] = q.z; x[3] = q.w;
    } else {
#pragma unroll
        for (int j = 0; j < NI; ++j) x[j] = p[j * IS];
    }
}

// out[b][.. o ..] = sum_j M[o][j] in[b][.. j ..] along direction D, o < MO
// (M row-major with row stride MAXNP, indexed at compile time)
template <int NB, int A0, int A1, int A2, int D, int MO, typename Real>
__device__ __forceinline__ void red_lines(const Real* in, Real* out, const Real (&M)[MAXNP * MAXNP], int lane) {
    using L = LineMap<A0, A1, A2, D, MO>;
    constexpr int NT = NB * L::NL;
#pragma unroll
    for (int it = 0; it < (NT + 31) / 32; ++it) {
        const int t = lane + 32 * it;
        if (NT % 32 != 0 && t >= NT) break;
        const int b = t / L::NL, r = t - b * L::NL;
        Real x[L::NI];
        red_ld<L::NI, L::IS>(in + L::ib(b, r), x);
        Real* o = out + L::ob(b, r);
        Real y[MO];
#pragma unroll
        for (int i = 0; i < MO; ++i) {
            Real a = Real(0);
#pragma unroll
            for (int j = 0; j < L::NI; ++j) a = fma_rn(M[i * MAXNP + j], x[j], a);
            y[i] = a;
        }
        if constexpr (MO == 4 && L::OS == 1 && sizeof(Real) == 4) {
            *reinterpret_cast<float4*>(o) = make_float4(y[0], y[1], y[2], y[3]);
        } else {
#pragma unroll
            for (int i = 0; i < MO; ++i) o[i * L::OS] = y[i];
        }
    }
}

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

// face normals of the lane's face points (Nr[d][it]: face 2d + side,
// t = lane + 32 it, side = t >= NFP)
template <int DIM, int NFP, int NFI, typename Real>
__device__ __forceinline__ void red_normals(const Geo<Real>& g, int64_t e, Real (&Nr)[DIM][NFI][DIM], int lane) {
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
        for (int it = 0; it < NFI; ++it) {
            const int t = lane + 32 * it;
            const int side = t >= NFP ? 1 : 0;
            if (t < 2 * NFP) load_normal<DIM>(g, e, 2 * d + side, t - side * NFP, Nr[d][it]);
        }
}

// One face array from NI to NO points per face direction: out = M (x) M in
// (M [NO][NI], both face directions in 3D); in with unit stride, out with
// unit stride
template <int DIM, int NI, int NO, typename Real>
__device__ __forceinline__ void red_face_map(const Real* in, Real* out, const Real (&M)[MAXNP * MAXNP]) {
    constexpr int NFI = DIM == 2 ? NI : NI * NI;
    Real x[NFI];
#pragma unroll
    for (int j = 0; j < NFI; ++j) x[j] = in[j];
    if constexpr (DIM == 2) {
#pragma unroll
        for (int a = 0; a < NO; ++a) {
            Real s = Real(0);
#pragma unroll
            for (int j = 0; j < NI; ++j) s = fma_rn(M[a * MAXNP + j], x[j], s);
            out[a] = s;
        }
    } else {
        Real t[NO][NI];   // along a, for every input b
#pragma unroll
        for (int a = 0; a < NO; ++a)
#pragma unroll
            for (int jb = 0; jb < NI; ++jb) {
                Real s = Real(0);
#pragma unroll
                for (int j = 0; j < NI; ++j) s = fma_rn(M[a * MAXNP + j], x[j + NI * jb], s);
                t[a][jb] = s;
            }
#pragma unroll
        for (int b = 0; b < NO; ++b)
#pragma unroll
            for (int a = 0; a < NO; ++a) {
                Real s = Real(0);
#pragma unroll
                for (int jb = 0; jb < NI; ++jb) s = fma_rn(M[b * MAXNP + jb], t[a][jb], s);
                out[a + NO * b] = s;
            }
    }
}

// the neighbour codes of element e, in every lane
template <int NF, typename Real>
__device__ __forceinline__ void red_codes_of(const Geo<Real>& g, int64_t e, int (&codes)[NF], int lane) {
    const int mine = lane < NF ? g.nbr[e * NF + lane] : 0;
#pragma unroll
    for (int f = 0; f < NF; ++f) codes[f] = __shfl_sync(0xffffffffu, mine, f);
}


// u at the Q points from the state at the P points (Iqp along every
// direction); y: scratch of RedSz::NYS values
template <int DIM, int NP, int NQ, typename Real>
__device__ __forceinline__ void red_to_q(const Real* su, Real* y, Real* uq, const Red<Real>& rd, int lane) {
    constexpr int NV = DIM + 2;
    if constexpr (DIM == 2) {
        red_lines<NV, NP, NP, 1, 0, NQ>(su, y, rd.Iqp, lane);
        __syncwarp();
        red_lines<NV, NQ, NP, 1, 1, NQ>(y, uq, rd.Iqp, lane);
    } else {
        constexpr int YB = red_al(NV * NP * NP * NQ);
        red_lines<NV, NP, NP, NP, 0, NQ>(su, y, rd.Iqp, lane);
        __syncwarp();
        red_lines<NV, NQ, NP, NP, 1, NQ>(y, y + YB, rd.Iqp, lane);
        __syncwarp();
        red_lines<NV, NQ, NQ, NP, 2, NQ>(y + YB, uq, rd.Iqp, lane);
    }
    __syncwarp();
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
    constexpr int NV = RS::NV, NP = RS::NP, NSP = RS::NSP, NFP = RS::NFP, NF = RS::NF;
    constexpr int NQ = RS::NQ, NSQ = RS::NSQ, NFQ = RS::NFQ, RW = RS::RW;
    constexpr int W = red_w<DIM, P, Q, Real>(true);
    constexpr int NFI = (2 * NFP + 31) / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int k = blockIdx.x * W + warp;
    if (k >= rd.n) return;
    Real* base = reinterpret_cast<Real*>(smem) + warp * RS::f_total;
    Real* su = base + RS::f_su;
    Real* sm = base + RS::f_sm;   // jumps [NF*NV][RW] at the P face points, then scratch, q_d, gradient
    Real* jq = base + RS::f_jq;   // projected jumps [NF][NV][NFQ]
    Real* uq = base + RS::f_uq;
    Real* gq = base + RS::f_gq;   // G at the Q face points of the two faces of one direction
    Real* gp = base + RS::f_gp;   // ... at their P face points, [2][NV][DIM][RW]
    const int64_t e = rd.elem[k];
    const Real* Sk = rd.S + int64_t(k) * rd.sS;    // S [DIM*DIM][NSQ] at the Q points
    const Real* iJk = rd.iJ + int64_t(k) * rd.sJ;  // 1/|J| [NSQ]
    const Real* ufe = uf + e * RS::FA;
    int codes[NF];
    red_codes_of<NF>(g, e, codes, lane);
    warp_stage_auto<NV * NSP, true>(su, u + e * NV * NSP, lane);
    cp_async_commit();
    // jumps u_c - u_f at the degree-P face points
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
        for (int it = 0; it < NFI; ++it) {
            const int t = lane + 32 * it;
            if ((2 * NFP) % 32 != 0 && t >= 2 * NFP) break;
            const int side = t >= NFP ? 1 : 0, fp = t - side * NFP, f = 2 * d + side;
            const int code = side ? codes[2 * d + 1] : codes[2 * d];
            Real uL[NV], uc[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) uL[v] = ufe[(f * NV + v) * NFP + fp];
            if (code >= 0) {
                const Real* un = uf + int64_t(code >> 3) * NV * NFP + omap<DIM, NP>(code & 7, fp);
#pragma unroll
                for (int v = 0; v < NV; ++v) uc[v] = Real(0.5) * (uL[v] + un[v * NFP]);
            } else {
                Real N[DIM], ug[NV];
                load_normal<DIM>(g, e, f, fp, N);
                bc_state<DIM>(-code, uL, N, ph, ug, uc);
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) sm[(f * NV + v) * RW + fp] = uc[v] - uL[v];
        }
    cp_async_wait<0>();
    __syncwarp();
    // mortar of the jumps
#pragma unroll
    for (int it = 0; it < (NF * NV + 31) / 32; ++it) {
        const int t = lane + 32 * it;
        if ((NF * NV) % 32 != 0 && t >= NF * NV) break;
        red_face_map<DIM, NP, NQ>(sm + t * RW, jq + t * NFQ, rd.Pqp);
    }
    __syncwarp();
    red_to_q<DIM, NP, NQ>(su, sm, uq, rd, lane);
    // reference derivatives q_d of u_q along each direction, [DIM][NV][NSQ]
    red_for<0, DIM>([&](auto dc) {
        constexpr int d = decltype(dc)::value;
        using L = LineMap<NQ, NQ, DIM == 2 ? 1 : NQ, d, NQ>;
        constexpr int NT = NV * NFQ;
#pragma unroll
        for (int it = 0; it < (NT + 31) / 32; ++it) {
            const int t = lane + 32 * it;
            if (NT % 32 != 0 && t >= NT) break;
            const int v = t / NFQ, r = t - v * NFQ;
            Real x[NQ];
            red_ld<NQ, L::IS>(uq + L::ib(v, r), x);
            Real* o = sm + d * NV * NSQ + L::ib(v, r);
#pragma unroll
            for (int i = 0; i < NQ; ++i) {
                Real a = Real(0);
#pragma unroll
                for (int j = 0; j < NQ; ++j) a = fma_rn(rd.D[i * MAXNP + j], x[j], a);
                o[i * L::IS] = a;
            }
        }
    });
    __syncwarp();
    // physical gradient at the Q points, (1/|J|) S^T q, in place
#pragma unroll
    for (int it = 0; it < (NSQ + 31) / 32; ++it) {
        const int pt = lane + 32 * it;
        if (NSQ % 32 != 0 && pt >= NSQ) break;
        Real S[DIM * DIM];
#pragma unroll
        for (int kk = 0; kk < DIM * DIM; ++kk) S[kk] = Sk[kk * NSQ + pt];
        const Real iJ = iJk[pt];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            Real qd[DIM];
#pragma unroll
            for (int d = 0; d < DIM; ++d) qd[d] = sm[(d * NV + v) * NSQ + pt];
#pragma unroll
            for (int i = 0; i < DIM; ++i) {
                Real a = Real(0);
#pragma unroll
                for (int d = 0; d < DIM; ++d) a += S[d * DIM + i] * qd[d];
                sm[(i * NV + v) * NSQ + pt] = a * iJ;
            }
        }
    }
    __syncwarp();
    red_for<0, DIM>([&](auto dc) {
        constexpr int d = decltype(dc)::value;
        using L = LineMap<NQ, NQ, DIM == 2 ? 1 : NQ, d, NQ>;
        // G at the Q face points of faces 2d, 2d + 1: the line's end value of
        // the gradient plus eta times the face's lifting, lc_i (u_c - u_f)
        // with lc_i = nsign sum_j l_j(+-1) h_j (S[d][i] / |J|)(x_j)
        constexpr int NT = 2 * NFQ;
#pragma unroll
        for (int it = 0; it < (NT + 31) / 32; ++it) {
            const int t = lane + 32 * it;
            if (NT % 32 != 0 && t >= NT) break;
            const int s = t >= NFQ ? 1 : 0, r = t - s * NFQ, f = 2 * d + s;
            const int b0 = L::ib(0, r);
            const Real nsg = s ? Real(1) : Real(-1);
            Real lv[NQ], hl[NQ];
#pragma unroll
            for (int j = 0; j < NQ; ++j) {
                lv[j] = s ? rd.lp[j] : rd.lm[j];
                hl[j] = lv[j] * (s ? rd.hp[j] : rd.hm[j]);
            }
            Real lc[DIM];
#pragma unroll
            for (int i = 0; i < DIM; ++i) {
                Real a = Real(0);
#pragma unroll
                for (int j = 0; j < NQ; ++j) {
                    const int pt = b0 + j * L::IS;
                    a += hl[j] * (nsg * (Sk[(d * DIM + i) * NSQ + pt] * iJk[pt]));
                }
                lc[i] = ph.eta * a;
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const Real jv = jq[(f * NV + v) * NFQ + r];
#pragma unroll
                for (int i = 0; i < DIM; ++i) {
                    Real a = Real(0);
#pragma unroll
                    for (int j = 0; j < NQ; ++j) a += lv[j] * sm[(i * NV + v) * NSQ + b0 + j * L::IS];
                    gq[((s * NV + v) * DIM + i) * NFQ + r] = a + lc[i] * jv;
                }
            }
        }
        __syncwarp();
        // G at the degree-P face points
        constexpr int NR = 2 * NV * DIM;
#pragma unroll
        for (int it = 0; it < (NR + 31) / 32; ++it) {
            const int t = lane + 32 * it;
            if (NR % 32 != 0 && t >= NR) break;
            red_face_map<DIM, NQ, NP>(gq + t * NFQ, gp + t * RW, rd.Ipq);
        }
        __syncwarp();
        // viscous normal fluxes there
#pragma unroll
        for (int it = 0; it < NFI; ++it) {
            const int t = lane + 32 * it;
            if ((2 * NFP) % 32 != 0 && t >= 2 * NFP) break;
            const int side = t >= NFP ? 1 : 0, fp = t - side * NFP, f = 2 * d + side;
            const int code = side ? codes[2 * d + 1] : codes[2 * d];
            Real G[NV][DIM], uL[NV], Fn[NV], N[DIM];
            load_normal<DIM>(g, e, f, fp, N);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                uL[v] = ufe[(f * NV + v) * NFP + fp];
#pragma unroll
                for (int i = 0; i < DIM; ++i) G[v][i] = gp[((side * NV + v) * DIM + i) * RW + fp];
            }
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
        }
        __syncwarp();
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
    constexpr int NQ = RS::NQ, NSQ = RS::NSQ, NFQ = RS::NFQ, FA = RS::FA, RW = RS::RW;
    constexpr int W = red_w<DIM, P, Q, Real>(false);
    constexpr int NFI = (2 * NFP + 31) / 32;
    constexpr int NL = NV * NFP;              // lines of the last direction (final pass)
    constexpr int NLI = (NL + 31) / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int k = blockIdx.x * W + warp;
    if (k >= rd.n) return;
    Real* base = reinterpret_cast<Real*>(smem) + warp * RS::total;
    Real* su = base + RS::su;
    Real* sm = base + RS::sm;     // jumps, then common fluxes [2*NF*NV][RW]; then scratch, q_d, F~_d
    Real* jf = base + RS::sjf;    // projected jumps [NF][NV][NFQ], then fluxes
    Real* uq = base + RS::suq;    // u_q, then R_q
    const int64_t e = rd.elem[k];
    const Real* Sk = rd.S + int64_t(k) * rd.sS;
    const Real* iJk = rd.iJ + int64_t(k) * rd.sJ;
    const Real* ufe = uf + e * FA;
    int codes[NF];
    red_codes_of<NF>(g, e, codes, lane);
    warp_stage_auto<NV * NSP, true>(su, u + e * NV * NSP, lane);
    cp_async_commit();
    // common normal flux (Rusanov minus the common viscous flux) and jump at
    // the degree-P face points
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
        for (int it = 0; it < NFI; ++it) {
            const int t = lane + 32 * it;
            if ((2 * NFP) % 32 != 0 && t >= 2 * NFP) break;
            const int side = t >= NFP ? 1 : 0, fp = t - side * NFP, f = 2 * d + side;
            const int code = side ? codes[2 * d + 1] : codes[2 * d];
            Real N[DIM], uL[NV], uR[NV], uc[NV];
            load_normal<DIM>(g, e, f, fp, N);
#pragma unroll
            for (int v = 0; v < NV; ++v) uL[v] = ufe[(f * NV + v) * NFP + fp];
            int64_t nb = 0;
            if (code >= 0) {
                nb = int64_t(code >> 3) * NV * NFP + omap<DIM, NP>(code & 7, fp);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    uR[v] = uf[nb + v * NFP];
                    uc[v] = Real(0.5) * (uL[v] + uR[v]);
                }
            } else {
                bc_state<DIM>(-code, uL, N, ph, uR, uc);
            }
            Real Fc[NV];
            rusanov<DIM>(uL, uR, N, ph.gamma, ph.gm1, Fc);
            if constexpr (VISC) {
                const Real* own = fvn + (e * NF + f) * NV * NFP + fp;
                if (code >= 0) {
#pragma unroll
                    for (int v = 0; v < NV; ++v) Fc[v] -= Real(0.5) * (own[v * NFP] - fvn[nb + v * NFP]);
                } else {
#pragma unroll
                    for (int v = 0; v < NV; ++v) Fc[v] -= own[v * NFP];
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                sm[(f * NV + v) * RW + fp] = uc[v] - uL[v];
                sm[((NF + f) * NV + v) * RW + fp] = Fc[v];
            }
        }
    cp_async_wait<0>();
    __syncwarp();
    // mortar of the jumps and fluxes
#pragma unroll
    for (int it = 0; it < (2 * NF * NV + 31) / 32; ++it) {
        const int t = lane + 32 * it;
        if ((2 * NF * NV) % 32 != 0 && t >= 2 * NF * NV) break;
        red_face_map<DIM, NP, NQ>(sm + t * RW, jf + t * NFQ, rd.Pqp);
    }
    __syncwarp();
    red_to_q<DIM, NP, NQ>(su, sm, uq, rd, lane);
    const Real* jq = jf;
    const Real* fq = jf + NF * NV * NFQ;
    // corrected gradient q_d = D_d u_q + g' terms of the projected jumps
    if constexpr (VISC) {
        red_for<0, DIM>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            using L = LineMap<NQ, NQ, DIM == 2 ? 1 : NQ, d, NQ>;
            constexpr int NT = NV * NFQ;
#pragma unroll
            for (int it = 0; it < (NT + 31) / 32; ++it) {
                const int t = lane + 32 * it;
                if (NT % 32 != 0 && t >= NT) break;
                const int v = t / NFQ, r = t - v * NFQ;
                Real x[NQ];
                red_ld<NQ, L::IS>(uq + L::ib(v, r), x);
                const Real jm = jq[((2 * d) * NV + v) * NFQ + r];
                const Real jp = jq[((2 * d + 1) * NV + v) * NFQ + r];
                Real* o = sm + d * NV * NSQ + L::ib(v, r);
#pragma unroll
                for (int i = 0; i < NQ; ++i) {
                    Real a = Real(0);
#pragma unroll
                    for (int j = 0; j < NQ; ++j) a += rd.D[i * MAXNP + j] * x[j];
                    o[i * L::IS] = a + rd.hp[i] * jp - rd.hm[i] * jm;
                }
            }
        });
        __syncwarp();
    }
    // flux at the Q points: F~_d = sum_i S[d][i] (F_inv - F_vis)_i (in place
    // of q_d)
#pragma unroll
    for (int it = 0; it < (NSQ + 31) / 32; ++it) {
        const int pt = lane + 32 * it;
        if (NSQ % 32 != 0 && pt >= NSQ) break;
        Real S[DIM * DIM], uu[NV], F[NV][DIM];
#pragma unroll
        for (int kk = 0; kk < DIM * DIM; ++kk) S[kk] = Sk[kk * NSQ + pt];
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
            const Real iJ = iJk[pt];
            Real G[NV][DIM];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                Real qd[DIM];
#pragma unroll
                for (int d = 0; d < DIM; ++d) qd[d] = sm[(d * NV + v) * NSQ + pt];
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
#pragma unroll
        for (int d = 0; d < DIM; ++d)
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                Real a = Real(0);
#pragma unroll
                for (int i = 0; i < DIM; ++i) a += S[d * DIM + i] * F[v][i];
                sm[(d * NV + v) * NSQ + pt] = a;
            }
    }
    __syncwarp();
    // divergence plus correction, one direction after the other, then
    // R_q = -div / |J| (in place of u_q)
    red_for<0, DIM>([&](auto dc) {
        constexpr int d = decltype(dc)::value;
        using L = LineMap<NQ, NQ, DIM == 2 ? 1 : NQ, d, NQ>;
        constexpr int NT = NV * NFQ;
#pragma unroll
        for (int it = 0; it < (NT + 31) / 32; ++it) {
            const int t = lane + 32 * it;
            if (NT % 32 != 0 && t >= NT) break;
            const int v = t / NFQ, r = t - v * NFQ;
            const int b0 = L::ib(0, r);
            Real x[NQ];
            red_ld<NQ, L::IS>(sm + d * NV * NSQ + v * NSQ + b0, x);
            Real em = Real(0), ep = Real(0);
#pragma unroll
            for (int j = 0; j < NQ; ++j) {
                em += rd.lm[j] * x[j];
                ep += rd.lp[j] * x[j];
            }
            const Real cm = fq[((2 * d) * NV + v) * NFQ + r] + em;   // Fc.N - (-1) I_-[F~_d]
            const Real cp = fq[((2 * d + 1) * NV + v) * NFQ + r] - ep;
#pragma unroll
            for (int i = 0; i < NQ; ++i) {
                Real a = Real(0);
#pragma unroll
                for (int j = 0; j < NQ; ++j) a += rd.D[i * MAXNP + j] * x[j];
                a += rd.hm[i] * cm + rd.hp[i] * cp;
                const int pt = b0 + i * L::IS;
                Real* o = uq + v * NSQ + pt;
                if constexpr (d == 0) *o = a;
                else if constexpr (d < DIM - 1) *o += a;
                else *o = -(*o + a) * iJk[pt];
            }
        }
        __syncwarp();
    });
    // R at the degree-P points: the passes along the first directions into
    // scratch, the last one fused with the stage update and the traces on the
    // two faces of the last direction
    if constexpr (DIM == 2) {
        red_lines<NV, NQ, NQ, 1, 0, NP>(uq, sm, rd.Ipq, lane);
    } else {
        red_lines<NV, NQ, NQ, NQ, 0, NP>(uq, sm + RS::YB, rd.Ipq, lane);
        __syncwarp();
        red_lines<NV, NP, NQ, NQ, 1, NP>(sm + RS::YB, sm, rd.Ipq, lane);
    }
    __syncwarp();
    const Real dt = st.dte ? st.dte[e] : st.dt;
    bool bad = false;
    constexpr int LD = DIM - 1;
    const int64_t eb = e * NV * NSP;
    {
        using LI = LineMap<NP, DIM == 2 ? NQ : NP, DIM == 2 ? 1 : NQ, LD, NP>;   // R along the last direction
        using LF = LineMap<NP, NP, DIM == 2 ? 1 : NP, LD, NP>;                   // the P points
        Real* ufn = st.uf_next ? st.uf_next + e * FA : nullptr;
#pragma unroll
        for (int it = 0; it < NLI; ++it) {
            const int t = lane + 32 * it;
            if (NL % 32 != 0 && t >= NL) break;
            const int v = t / NFP, r = t - v * NFP;
            const int b0 = LF::ib(v, r);
            Real pu0[NP], pacc[NP];
            if (st.stage >= 2) {
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    pu0[i] = st.u0[eb + b0 + i * LF::IS];
                    pacc[i] = st.acc[eb + b0 + i * LF::IS];
                }
            }
            Real x[NQ];
            red_ld<NQ, LI::IS>(sm + LI::ib(v, r), x);
            Real nu[NP];
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                Real a = Real(0);
#pragma unroll
                for (int j = 0; j < NQ; ++j) a = fma_rn(rd.Ipq[i * MAXNP + j], x[j], a);
                const int o = b0 + i * LF::IS;
                nu[i] = red_stage(st, dt, a, su[o], pu0[i], pacc[i], eb + o, bad);
                su[o] = nu[i];
            }
            if (ufn) {
                Real tm = Real(0), tp = Real(0);
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    tm += op.lm[j] * nu[j];
                    tp += op.lp[j] * nu[j];
                }
                ufn[((2 * LD) * NV + v) * NFP + r] = tm;
                ufn[((2 * LD + 1) * NV + v) * NFP + r] = tp;
            }
        }
    }
    if (st.nonfinite && __any_sync(0xffffffffu, bad) && lane == 0) {
        int c = 0;
        while (c + 1 < st.ncand && e >= st.cand_off[c + 1]) ++c;
        atomicOr(st.nonfinite + c, 1);
    }
    if (st.uf_next) {
        __syncwarp();
        // traces of the new state on the faces of the other directions
        Real* ufn = st.uf_next + e * FA;
        red_for<0, LD>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            using L = LineMap<NP, NP, DIM == 2 ? 1 : NP, d, NP>;
#pragma unroll
            for (int it = 0; it < NLI; ++it) {
                const int t = lane + 32 * it;
                if (NL % 32 != 0 && t >= NL) break;
                const int v = t / NFP, r = t - v * NFP;
                Real x[NP];
                red_ld<NP, L::IS>(su + L::ib(v, r), x);
                Real tm = Real(0), tp = Real(0);
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    tm += op.lm[j] * x[j];
                    tp += op.lp[j] * x[j];
                }
                ufn[((2 * d) * NV + v) * NFP + r] = tm;
                ufn[((2 * d + 1) * NV + v) * NFP + r] = tp;
            }
        });
    }
}

}  // namespace frk
