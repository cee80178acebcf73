// libfr C-ABI: context set-up (mesh preprocessing in double on the host),
// state management, residual / RK4 step launch sequences, CUDA-graph replay,
// forces, volume integrals and FW-H surface sampling.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "fr.h"
#include "fr_common.h"
#include "fr_geom.h"

static thread_local std::string g_err;

static int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define CK(x)                                                                                   \
    do {                                                                                        \
        cudaError_t e_ = (x);                                                                   \
        if (e_ != cudaSuccess) return fail(FR_ECUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CKL(rc, what)                                                                          \
    do {                                                                                       \
        if ((rc) != 0)                                                                         \
            return fail(FR_ECUDA, std::string(what) + ": " + cudaGetErrorString(cudaError_t(rc))); \
    } while (0)

namespace {

struct Surface {
    int cand = 0, npts = 0, cap = 0, every = 1;
    int64_t* pe = nullptr;   // element of each point (global index)
    void* pw = nullptr;      // 1D Lagrange weights [npts][dim][np]
    void* hist = nullptr;    // [cap][npts][5] deviations from the free stream
    int* count = nullptr;    // device int[3]: records, steps seen, overflow flag
};

}  // namespace

struct fr_ctx {
    int dim = 0, p = 0, np = 0, nsp = 0, nfp = 0, nf = 0, nv = 0;
    int ncand = 0, prec = 0, visc = 0, kind = 0, affine = 0, diag = 0, bnd = 1;
    int64_t E = 0;
    fr_options opt{};
    std::vector<int64_t> cand_off;
    std::vector<std::vector<double>> nodes;  // per candidate
    std::vector<int> q;                      // per candidate geometry order
    frg::Ref1D ref{};
    size_t rsz = 8;                          // sizeof(Real)
    // device buffers
    void *u0 = nullptr, *us = nullptr, *acc = nullptr, *fvn = nullptr;
    void* ufb[2] = {nullptr, nullptr};   // ping-pong flux-point traces
    bool traces_valid = false;           // ufb[0] holds the traces of u0
    void *S = nullptr, *J = nullptr, *iJ = nullptr, *N = nullptr;
    frk::Ops<double> opd{};
    frk::Ops<float> opf{};
    int32_t* nbr = nullptr;
    int64_t sS_e = 0, sS_k = 0, sS_sp = 0, sJ_e = 0, sJ_sp = 0, sN_f = 0, sN_fp = 0;
    int32_t* wall_ef = nullptr;
    int64_t* wall_off_d = nullptr;
    std::vector<int64_t> wall_off;
    double *fnow = nullptr, *fsum = nullptr, *fcnt = nullptr, *partial = nullptr, *fpart = nullptr;
    int partial_blocks = 0;
    std::vector<Surface> surf;
    frk::Launch lc[3]{};
    cudaStream_t cap_stream = nullptr;
    // the reduced-degree kernels of a step run on red_stream[q] (one per
    // degree q), forked from the step's stream and joined back (they write
    // only the reduced elements' arrays, the degree-p kernels only the others')
    cudaStream_t red_stream[frk::MAXNP] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[frk::MAXNP] = {};
    cudaGraphExec_t gexec = nullptr;
    int64_t launches = 0;
    int64_t graph_launches_per_step = 0;
    int device = 0;
    double* stage64 = nullptr;  // double staging buffer for FP32 state transfers
    void* dte = nullptr;        // per-element time step (Real[E]) once a candidate sets its own
    std::vector<double> cand_dt;  // per-candidate step (host copy)
    // energy sources (Appendix D, Eq. D.1), see frk::Src
    std::vector<std::vector<std::array<double, 6>>> srcs;  // per candidate: A, k, x, y, z, f
    int src_nentry = 0;            // elements that carry a source (0: none)
    int32_t* src_elem = nullptr;   // device [entries]
    int32_t* src_cand = nullptr;   // device [entries]
    void* src_w = nullptr;         // device Real [entries][MAXSRC][nsp]
    double *src_A = nullptr, *src_f = nullptr;  // device [ncand][MAXSRC]
    double* tnow = nullptr;        // device [ncand]: time at the start of the next step
    double* dtc = nullptr;         // device [ncand]: step of each candidate
    // adaptive time step (cfl > 0: on)
    double adaptive_cfl = 0.0;
    void* hlen = nullptr;                // device Real [E]: element length
    int64_t* cand_off_d = nullptr;       // device [ncand + 1]
    unsigned long long* lam = nullptr;   // device [ncand]: max spectral rate (double bits)
    // variable polynomial order (sponge zones), see frk::Sponge
    std::vector<std::vector<int32_t>> order;  // per candidate: [count] degree caps (empty: all p)
    int sp_n = 0;                             // capped elements (0: none)
    int32_t *sp_elem = nullptr, *sp_cap = nullptr;  // device [sp_n]
    std::vector<int> sp_off;                  // [ncand + 1]: each candidate's slice of the list
    // the reduced elements grouped by degree q < p for the kernels of frk::Red:
    // device lists, metric terms at their q points, per-element degrees
    int red_n[frk::MAXNP] = {0, 0, 0, 0, 0};
    int32_t* red_elem[frk::MAXNP] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    void* red_S[frk::MAXNP] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    void* red_iJ[frk::MAXNP] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    signed char* order_d = nullptr;           // device [E] (null: no reduced element)
    // non-finite state detection: nonfinite[c] != 0 once candidate c's state
    // held a NaN or an infinity at the end of a step (cleared by fr_state_set)
    int* nonfinite = nullptr;                 // device [ncand]
    // explicit scheme in coefficient form (empty: classic RK4), per stage
    // (a, b, c, d, e, f); ls_time[i] = abscissa of stage i's input (in dt)
    std::vector<std::array<double, 6>> lsc;
    std::vector<double> ls_time;
    void* ufb3 = nullptr;                     // third trace buffer (odd stage counts)
};

namespace {

template <typename Real>
frk::Src<Real> src_of(const fr_ctx* c, double cfac) {
    frk::Src<Real> r;
    if (c->src_nentry <= 0) return r;
    r.nentry = c->src_nentry;
    r.elem = c->src_elem;
    r.cand = c->src_cand;
    r.w = static_cast<const Real*>(c->src_w);
    r.A = c->src_A;
    r.f = c->src_f;
    r.tnow = c->tnow;
    r.cfac = cfac;
    return r;
}

__global__ void k_time_advance(double* __restrict__ tnow, const double* __restrict__ dtc, int ncand) {
    for (int c = threadIdx.x; c < ncand; c += blockDim.x) tnow[c] += dtc[c];
}

// adaptive step of each candidate, dt = cfl / lambda_max, into the per-element
// step and the per-candidate step
template <typename Real>
__global__ void k_dt_fill(const unsigned long long* __restrict__ lam, double cfl, const int64_t* __restrict__ cand_off,
                          int ncand, int64_t E, Real* __restrict__ dte, double* __restrict__ dtc) {
    for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < E; e += int64_t(gridDim.x) * blockDim.x) {
        int c = 0;
        while (c + 1 < ncand && e >= cand_off[c + 1]) ++c;
        const double dt = cfl / __longlong_as_double(static_cast<long long>(lam[c]));
        dte[e] = Real(dt);
        if (e == cand_off[c]) dtc[c] = dt;
    }
}


template <typename Real>
frk::Geo<Real> geo_of(const fr_ctx* c) {
    frk::Geo<Real> g;
    g.S = static_cast<const Real*>(c->S);
    g.J = static_cast<const Real*>(c->J);
    g.iJ = static_cast<const Real*>(c->iJ);
    g.N = static_cast<const Real*>(c->N);
    g.nbr = c->nbr;
    g.sS_e = c->sS_e;
    g.sS_k = c->sS_k;
    g.sS_sp = c->sS_sp;
    g.sJ_e = c->sJ_e;
    g.sJ_sp = c->sJ_sp;
    g.sN_f = c->sN_f;
    g.sN_fp = c->sN_fp;
    g.diag = c->diag;
    g.bnd = c->bnd;
    g.order = c->order_d;
    return g;
}

template <typename Real>
const frk::Ops<Real>& ops_ref(const fr_ctx* c);
template <>
const frk::Ops<double>& ops_ref<double>(const fr_ctx* c) { return c->opd; }
template <>
const frk::Ops<float>& ops_ref<float>(const fr_ctx* c) { return c->opf; }

template <typename Real>
frk::Phys<Real> phys_of(const fr_ctx* c) {
    frk::Phys<Real> ph;
    const fr_options& o = c->opt;
    ph.gamma = Real(o.gamma);
    ph.gm1 = Real(o.gamma - 1.0);
    ph.mu = Real(o.mu);
    ph.kappa = Real(o.mu * o.gamma / o.prandtl);
    ph.eta = Real(o.br2_eta);
    ph.rho_inf = Real(o.rho_inf);
    ph.p_inf = Real(o.p_inf);
    for (int i = 0; i < 3; ++i) ph.vel_inf[i] = Real(o.vel_inf[i]);
    ph.viscous = c->visc;
    return ph;
}

template <typename Real>
frk::Ops<Real> ops_of(const frg::Ref1D& r) {
    frk::Ops<Real> op;
    std::memset(&op, 0, sizeof(op));
    double lhm = 0, lhp = 0;
    for (int j = 0; j < r.np; ++j) {
        op.lm[j] = Real(r.lm[j]);
        op.lp[j] = Real(r.lp[j]);
        op.hm[j] = Real(r.hm[j]);
        op.hp[j] = Real(r.hp[j]);
        op.w[j] = Real(r.w[j]);
        op.dlm[j] = Real(frg::lagrange_deriv(r.x, r.np, j, -1.0));
        for (int k = 0; k < r.np; ++k) op.D[j * frk::MAXNP + k] = Real(r.D[j][k]);
        lhm += r.lm[j] * r.hm[j];
        lhp += r.lp[j] * r.hp[j];
    }
    op.lhm = Real(lhm);
    op.lhp = Real(lhp);
    return op;
}

// ---- dimension dispatch of the per-TU launchers
template <typename Real>
int L_traces(fr_ctx* c, const Real* u, Real* uf, cudaStream_t s) {
    const auto& op = ops_ref<Real>(c);
    ++c->launches;
    return c->dim == 2 ? frl::traces<Real, 2>(c->p, u, uf, c->E, op, c->lc[0], s)
                       : frl::traces<Real, 3>(c->p, u, uf, c->E, op, c->lc[0], s);
}

template <typename Real>
int L_visc(fr_ctx* c, const Real* u, const Real* uf, cudaStream_t s) {
    const auto& op = ops_ref<Real>(c);
    Real* fvn = static_cast<Real*>(c->fvn);
    const auto ph = phys_of<Real>(c);
    const auto g = geo_of<Real>(c);
    ++c->launches;
    return c->dim == 2 ? frl::visc_face<Real, 2>(c->p, u, uf, fvn, c->E, op, ph, g, c->lc[1], s)
                       : frl::visc_face<Real, 3>(c->p, u, uf, fvn, c->E, op, ph, g, c->lc[1], s);
}

template <typename Real>
int L_source(fr_ctx* c, const frk::Src<Real>& src, const frk::Stage<Real>& st, cudaStream_t s) {
    ++c->launches;
    const auto& op = ops_ref<Real>(c);
    return c->dim == 2 ? frl::source_stage<Real, 2>(c->p, src, st, op, s)
                       : frl::source_stage<Real, 3>(c->p, src, st, op, s);
}

// the 1D projections onto degree q = 0..p on the GL points,
// Pi_q[i][j] = sum_{k <= q} P_k(x_i) P_k(x_j) w_j (2k + 1) / 2
template <typename Real>
frk::Sponge<Real> sponge_of(const fr_ctx* c) {
    frk::Sponge<Real> r;
    r.n = c->sp_n;
    r.elem = c->sp_elem;
    r.cap = c->sp_cap;
    const int np = c->np;
    double L[frk::MAXNP][frk::MAXNP], dL[frk::MAXNP];
    for (int i = 0; i < np; ++i) frg::legendre(np - 1, c->ref.x[i], L[i], dL);
    for (int q = 0; q < frk::MAXNP; ++q)
        for (int i = 0; i < frk::MAXNP; ++i)
            for (int j = 0; j < frk::MAXNP; ++j) {
                double v = 0.0;
                if (i < np && j < np)
                    for (int k = 0; k <= q && k < np; ++k) v += L[i][k] * L[j][k] * c->ref.w[j] * (2 * k + 1) * 0.5;
                r.pm[q][i * frk::MAXNP + j] = Real(v);
            }
    return r;
}

// cand >= 0: that candidate's capped elements only
template <typename Real>
int L_sponge(fr_ctx* c, Real* a, Real* b, Real* uf_out, cudaStream_t s, int cand = -1) {
    if (c->sp_n <= 0) return 0;
    auto sp = sponge_of<Real>(c);
    if (cand >= 0) {
        sp.elem += c->sp_off[cand];
        sp.cap += c->sp_off[cand];
        sp.n = c->sp_off[cand + 1] - c->sp_off[cand];
        if (sp.n == 0) return 0;
    }
    ++c->launches;
    const auto& op = ops_ref<Real>(c);
    return c->dim == 2 ? frl::sponge<Real, 2>(c->p, sp, a, b, uf_out, op, s)
                       : frl::sponge<Real, 3>(c->p, sp, a, b, uf_out, op, s);
}

template <typename Real>
int L_resid(fr_ctx* c, const Real* u, const Real* uf, const frk::Stage<Real>& st, cudaStream_t s) {
    const auto& op = ops_ref<Real>(c);
    const Real* fvn = static_cast<const Real*>(c->fvn);
    const auto ph = phys_of<Real>(c);
    const auto g = geo_of<Real>(c);
    ++c->launches;
    if constexpr (sizeof(Real) == 4) {
        if (c->prec >= FR_TF32_TC)
            return frl::residual_tc3(c->p, c->prec == FR_TF32_TC ? 1 : 2, u, uf, fvn, c->E, op, ph, g, st, c->lc[2],
                                     s);
    }
    return c->dim == 2 ? frl::residual<Real, 2>(c->p, u, uf, fvn, c->E, op, ph, g, st, c->lc[2], s)
                       : frl::residual<Real, 3>(c->p, u, uf, fvn, c->E, op, ph, g, st, c->lc[2], s);
}

// the degree-q operators of the reduced elements (frk::Red): q = 0 takes the
// one linear correction function (DG), whatever the context's kind
template <typename Real>
frk::Red<Real> red_of(const fr_ctx* c, int q) {
    frk::Red<Real> r;
    std::memset(r.Iqp, 0, sizeof(r.Iqp));
    std::memset(r.Ipq, 0, sizeof(r.Ipq));
    std::memset(r.Pqp, 0, sizeof(r.Pqp));
    std::memset(r.D, 0, sizeof(r.D));
    std::memset(r.lm, 0, sizeof(r.lm));
    std::memset(r.lp, 0, sizeof(r.lp));
    std::memset(r.hm, 0, sizeof(r.hm));
    std::memset(r.hp, 0, sizeof(r.hp));
    frg::Ref1D rq;
    frg::build_ref(q, q > 0 ? c->kind : 0, rq);
    const frg::Ref1D& rp = c->ref;
    const int nq = q + 1, np = c->np;
    double Lq[frk::MAXNP][frk::MAXNP], Lp[frk::MAXNP][frk::MAXNP], dL[frk::MAXNP];
    for (int i = 0; i < nq; ++i) frg::legendre(q, rq.x[i], Lq[i], dL);
    for (int j = 0; j < np; ++j) frg::legendre(q, rp.x[j], Lp[j], dL);
    for (int i = 0; i < nq; ++i)
        for (int j = 0; j < np; ++j) {
            r.Iqp[i * frk::MAXNP + j] = Real(frg::lagrange(rp.x, np, j, rq.x[i]));
            r.Ipq[j * frk::MAXNP + i] = Real(frg::lagrange(rq.x, nq, i, rp.x[j]));
            double v = 0.0;
            for (int k = 0; k <= q; ++k) v += Lq[i][k] * Lp[j][k] * rp.w[j] * (2 * k + 1) * 0.5;
            r.Pqp[i * frk::MAXNP + j] = Real(v);
        }
    for (int i = 0; i < nq; ++i) {
        for (int j = 0; j < nq; ++j) r.D[i * frk::MAXNP + j] = Real(rq.D[i][j]);
        r.lm[i] = Real(rq.lm[i]);
        r.lp[i] = Real(rq.lp[i]);
        r.hm[i] = Real(rq.hm[i]);
        r.hp[i] = Real(rq.hp[i]);
    }
    const int nsq = c->dim == 2 ? nq * nq : nq * nq * nq;
    r.n = c->red_n[q];
    r.elem = c->red_elem[q];
    r.S = static_cast<const Real*>(c->red_S[q]);
    r.iJ = static_cast<const Real*>(c->red_iJ[q]);
    r.sS = int64_t(c->dim) * c->dim * nsq;
    r.sJ = nsq;
    return r;
}

template <typename Real>
int L_red_face(fr_ctx* c, int q, const Real* u, const Real* uf, cudaStream_t s) {
    if (c->red_n[q] <= 0) return 0;
    const auto rd = red_of<Real>(c, q);
    const auto& op = ops_ref<Real>(c);
    const auto ph = phys_of<Real>(c);
    const auto g = geo_of<Real>(c);
    Real* fvn = static_cast<Real*>(c->fvn);
    ++c->launches;
    return c->dim == 2 ? frl::red_face<Real, 2>(c->p, q, rd, u, uf, fvn, op, ph, g, s)
                       : frl::red_face<Real, 3>(c->p, q, rd, u, uf, fvn, op, ph, g, s);
}

template <typename Real>
int L_red_resid(fr_ctx* c, int q, const Real* u, const Real* uf, const frk::Stage<Real>& st, cudaStream_t s) {
    if (c->red_n[q] <= 0) return 0;
    const auto rd = red_of<Real>(c, q);
    const auto& op = ops_ref<Real>(c);
    const auto ph = phys_of<Real>(c);
    const auto g = geo_of<Real>(c);
    const Real* fvn = static_cast<const Real*>(c->fvn);
    ++c->launches;
    return c->dim == 2 ? frl::red_resid<Real, 2>(c->p, q, rd, u, uf, fvn, op, ph, g, st, s)
                       : frl::red_resid<Real, 3>(c->p, q, rd, u, uf, fvn, op, ph, g, st, s);
}

template <typename Real>
int L_forces(fr_ctx* c, cudaStream_t s) {
    if (c->wall_off.empty() || c->wall_off.back() == 0) return 0;
    const auto& op = ops_ref<Real>(c);
    const auto g = geo_of<Real>(c);
    const Real gm1 = Real(c->opt.gamma - 1.0);
    ++c->launches;
    return c->dim == 2
               ? frl::forces<Real, 2>(c->p, static_cast<const Real*>(c->ufb[0]), static_cast<const Real*>(c->fvn),
                                      c->wall_ef, c->wall_off_d, c->ncand, op, g, gm1, c->visc, c->fpart,
                                      c->fnow, c->fsum, c->fcnt, s)
               : frl::forces<Real, 3>(c->p, static_cast<const Real*>(c->ufb[0]), static_cast<const Real*>(c->fvn),
                                      c->wall_ef, c->wall_off_d, c->ncand, op, g, gm1, c->visc, c->fpart,
                                      c->fnow, c->fsum, c->fcnt, s);
}

template <typename Real>
int L_sample(fr_ctx* c, Surface& sf, cudaStream_t s) {
    const auto ph = phys_of<Real>(c);
    c->launches += 2;
    return c->dim == 2 ? frl::sample<Real, 2>(c->p, static_cast<const Real*>(c->u0), sf.pe,
                                              static_cast<const Real*>(sf.pw), sf.npts, ph,
                                              static_cast<Real*>(sf.hist), sf.count, sf.cap, sf.every, s)
                       : frl::sample<Real, 3>(c->p, static_cast<const Real*>(c->u0), sf.pe,
                                              static_cast<const Real*>(sf.pw), sf.npts, ph,
                                              static_cast<Real*>(sf.hist), sf.count, sf.cap, sf.every, s);
}

// Optional per-launch event pairs for fr_profile_step: kind 0..5.  With
// `external` set the records are made during stream capture and become event
// record nodes of the graph (re-recorded at every replay).
struct Prof {
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;
    cudaStream_t s = nullptr;
    bool external = false;
    void record(cudaEvent_t e) {
        if (external) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
        else cudaEventRecord(e, s);
    }
    void mark_begin(int k) {
        cudaEvent_t a;
        cudaEventCreate(&a);
        record(a);
        ev.push_back(a);
        kind.push_back(k);
    }
    void mark_end() {
        cudaEvent_t b;
        cudaEventCreate(&b);
        record(b);
        ev.push_back(b);
    }
};

// Traces of u0 into ufb[0] (needed once after the state changed from outside).
template <typename Real>
int ensure_traces(fr_ctx* c, cudaStream_t s, Prof* pr = nullptr) {
    if (c->traces_valid) return FR_OK;
    if (pr) pr->mark_begin(0);
    const int rc = L_traces<Real>(c, static_cast<const Real*>(c->u0), static_cast<Real*>(c->ufb[0]), s);
    if (pr) pr->mark_end();
    CKL(rc, "traces kernel");
    c->traces_valid = true;
    return FR_OK;
}

// One RK4 step; stage s reads the traces ufb[(s-1)&1] of its input and its
// residual kernel writes the traces of its output into ufb[s&1], so the step
// ends with the traces of the new u0 in ufb[0].
template <typename Real>
int enqueue_adaptive_dt(fr_ctx* c, cudaStream_t s) {
    CK(cudaMemsetAsync(c->lam, 0, sizeof(unsigned long long) * c->ncand, s));
    const auto ph = phys_of<Real>(c);
    const Real* u = static_cast<const Real*>(c->u0);
    const Real* h = static_cast<const Real*>(c->hlen);
    int rc = c->dim == 2 ? frl::cfl<Real, 2>(c->p, u, h, c->E, c->cand_off_d, c->ncand, ph, c->lam, s)
                         : frl::cfl<Real, 3>(c->p, u, h, c->E, c->cand_off_d, c->ncand, ph, c->lam, s);
    CKL(rc, "time step kernel");
    k_dt_fill<Real><<<256, 256, 0, s>>>(c->lam, c->adaptive_cfl, c->cand_off_d, c->ncand, c->E,
                                        static_cast<Real*>(c->dte), c->dtc);
    c->launches += 2;
    CK(cudaGetLastError());
    return FR_OK;
}

// the red streams wait for the work enqueued on s so far; s later waits for
// the work enqueued on them (inside a stream capture both become graph
// dependencies)
cudaError_t fork_red(fr_ctx* c, cudaStream_t s) {
    cudaError_t e = cudaEventRecord(c->ev_fork, s);
    for (int q = 0; q < c->p && e == cudaSuccess; ++q)
        if (c->red_n[q] > 0) e = cudaStreamWaitEvent(c->red_stream[q], c->ev_fork, 0);
    return e;
}
cudaError_t join_red(fr_ctx* c, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < c->p && e == cudaSuccess; ++q)
        if (c->red_n[q] > 0) {
            e = cudaEventRecord(c->ev_join[q], c->red_stream[q]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_join[q], 0);
        }
    return e;
}

template <typename Real>
int enqueue_step(fr_ctx* c, cudaStream_t s, Prof* pr = nullptr) {
    Real* u0 = static_cast<Real*>(c->u0);
    Real* us = static_cast<Real*>(c->us);
    Real* acc = static_cast<Real*>(c->acc);
    if (c->adaptive_cfl > 0.0) {
        const int rc = enqueue_adaptive_dt<Real>(c, s);
        if (rc) return rc;
    }
    // stage s reads the traces of its input and writes those of its output;
    // the step ends with the traces of the new u0 in ufb[0].  Even stage
    // counts alternate ufb[1], ufb[0]; odd ones alternate ufb[1], ufb3 and end
    // in ufb[0].
    const int ns = c->lsc.empty() ? 4 : int(c->lsc.size());
    auto trace_buf = [&](int st) -> Real* {
        if (st == 0 || st == ns) return static_cast<Real*>(c->ufb[0]);
        if (ns % 2 == 0) return static_cast<Real*>(c->ufb[st & 1]);
        return static_cast<Real*>(st & 1 ? c->ufb[1] : c->ufb3);
    };
    // reduced-degree kernels beside the degree-p ones (not when every launch
    // is timed on its own)
    bool fork = false;
    for (int q = 0; q < c->p; ++q) fork = fork || c->red_n[q] > 0;
    fork = fork && !pr;
    for (int stage = 1; stage <= ns; ++stage) {
        const Real* in = (stage == 1) ? u0 : us;
        const Real* uf_in = trace_buf(stage - 1);
        Real* uf_out = trace_buf(stage);
        int rc;
        if (c->visc) {
            // the reduced-degree kernels first: their few, latency-bound
            // blocks then start beside the degree-p kernel's
            if (fork) CK(fork_red(c, s));
            for (int q = 0; q < c->p; ++q)
                if (c->red_n[q] > 0) {
                    if (pr) pr->mark_begin(5);
                    rc = L_red_face<Real>(c, q, in, uf_in, fork ? c->red_stream[q] : s);
                    if (pr) pr->mark_end();
                    CKL(rc, "reduced-degree face kernel");
                }
            if (pr) pr->mark_begin(1);
            rc = L_visc<Real>(c, in, uf_in, s);
            if (pr) pr->mark_end();
            CKL(rc, "viscous face kernel");
            if (fork) CK(join_red(c, s));
        }
        if (stage == 1) {
            if (pr) pr->mark_begin(3);
            rc = L_forces<Real>(c, s);
            CKL(rc, "forces kernel");
            for (auto& sf : c->surf) {
                rc = L_sample<Real>(c, sf, s);
                CKL(rc, "sampling kernel");
            }
            if (pr) pr->mark_end();
        }
        frk::Stage<Real> st;
        st.stage = stage;
        st.dt = Real(c->opt.dt);
        st.dte = static_cast<const Real*>(c->dte);
        st.R = nullptr;
        st.u0 = u0;
        st.us = us;
        st.acc = acc;
        st.uf_next = uf_out;
        st.nonfinite = c->nonfinite;
        st.cand_off = c->cand_off_d;
        st.ncand = c->ncand;
        double cfac = stage == 1 ? 0.0 : stage == 4 ? 1.0 : 0.5;
        if (!c->lsc.empty()) {
            const auto& k = c->lsc[stage - 1];
            st.ls = 1;
            st.last = stage == ns;
            st.ca = Real(k[0]);
            st.cb = Real(k[1]);
            st.cc = Real(k[2]);
            st.cd = Real(k[3]);
            st.ce = Real(k[4]);
            st.cf = Real(k[5]);
            cfac = c->ls_time[stage - 1];
        }
        if (fork) CK(fork_red(c, s));
        for (int q = 0; q < c->p; ++q)
            if (c->red_n[q] > 0) {
                if (pr) pr->mark_begin(5);
                rc = L_red_resid<Real>(c, q, in, uf_in, st, fork ? c->red_stream[q] : s);
                if (pr) pr->mark_end();
                CKL(rc, "reduced-degree residual kernel");
            }
        if (pr) pr->mark_begin(2);
        rc = L_resid<Real>(c, in, uf_in, st, s);
        if (pr) pr->mark_end();
        CKL(rc, "residual kernel");
        if (fork) CK(join_red(c, s));
        if (c->src_nentry > 0) {
            if (pr) pr->mark_begin(4);
            rc = L_source<Real>(c, src_of<Real>(c, cfac), st, s);
            if (pr) pr->mark_end();
            CKL(rc, "source kernel");
        }
    }
    if (c->src_nentry > 0) {
        k_time_advance<<<1, 32, 0, s>>>(c->tnow, c->dtc, c->ncand);
        ++c->launches;
        CK(cudaGetLastError());
    }
    return FR_OK;
}

// One residual of a caller state u into R; uses ufb[0], so the traces of u0
// must be rebuilt before the next step.
template <typename Real>
int enqueue_residual(fr_ctx* c, const Real* u, Real* R, cudaStream_t s) {
    Real* uf = static_cast<Real*>(c->ufb[0]);
    c->traces_valid = false;
    int rc = L_traces<Real>(c, u, uf, s);
    CKL(rc, "traces kernel");
    if (c->visc) {
        rc = L_visc<Real>(c, u, uf, s);
        CKL(rc, "viscous face kernel");
        for (int q = 0; q < c->p; ++q) {
            rc = L_red_face<Real>(c, q, u, uf, s);
            CKL(rc, "reduced-degree face kernel");
        }
    }
    frk::Stage<Real> st;
    st.stage = 0;
    st.dt = Real(0);
    st.dte = nullptr;
    st.R = R;
    st.u0 = st.us = st.acc = st.uf_next = nullptr;
    rc = L_resid<Real>(c, u, uf, st, s);
    CKL(rc, "residual kernel");
    for (int q = 0; q < c->p; ++q) {
        rc = L_red_resid<Real>(c, q, u, uf, st, s);
        CKL(rc, "reduced-degree residual kernel");
    }
    if (c->src_nentry > 0) {
        rc = L_source<Real>(c, src_of<Real>(c, 0.0), st, s);
        CKL(rc, "source kernel");
    }
    return FR_OK;
}

// FP64 -> FP32 over n values; two values per 16-byte load when both arrays
// are aligned for it (the source may be host memory read over the CPU-GPU
// link, where wider requests move more bytes per request)
__global__ void k_d2f(const double* a, float* b, int64_t n) {
    const int64_t t0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x, st = int64_t(gridDim.x) * blockDim.x;
    if ((reinterpret_cast<uintptr_t>(a) & 15) == 0 && (reinterpret_cast<uintptr_t>(b) & 7) == 0) {
        const double2* a2 = reinterpret_cast<const double2*>(a);
        float2* b2 = reinterpret_cast<float2*>(b);
        for (int64_t i = t0; i < n / 2; i += st) {
            const double2 x = a2[i];
            b2[i] = make_float2(float(x.x), float(x.y));
        }
        if (t0 == 0 && (n & 1)) b[n - 1] = float(a[n - 1]);
    } else {
        for (int64_t i = t0; i < n; i += st) b[i] = float(a[i]);
    }
}
__global__ void k_f2d(const float* a, double* b, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        b[i] = double(a[i]);
}
__global__ void k_d2d(const double* a, double* b, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        b[i] = a[i];
}

// The address at which kernels on the current device reach host memory that
// the runtime has page-locked and mapped (cudaHostAlloc, cudaHostRegister: a
// pinned torch tensor, for instance), or nullptr for pageable memory.  State
// transfers from and to such memory convert in one kernel pass that reads or
// writes the host array directly over the CPU-GPU link, with no staging
// buffer and no separate copy.
const void* host_alias(const void* p) {
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
        cudaGetLastError();   // clear the error state a failed query leaves
        return nullptr;
    }
    return pa.type == cudaMemoryTypeHost ? pa.devicePointer : nullptr;
}

template <typename T>
int upload(void** dst, const std::vector<T>& src) {
    if (src.empty()) { *dst = nullptr; return FR_OK; }
    if (cudaMalloc(dst, src.size() * sizeof(T)) != cudaSuccess)
        return fail(FR_ENOMEM, "cudaMalloc failed for a mesh array");
    CK(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return FR_OK;
}

int upload_real(void** dst, const std::vector<double>& src, int prec) {
    if (prec == FR_FP64) return upload(dst, src);
    std::vector<float> f(src.begin(), src.end());
    return upload(dst, f);
}

int orient_map(int dim, int np, int o, int fp) {
    if (dim == 2) return (o & 1) ? np - 1 - fp : fp;
    int a = fp % np, b = fp / np;
    if (o & 4) std::swap(a, b);
    if (o & 1) a = np - 1 - a;
    if (o & 2) b = np - 1 - b;
    return a + np * b;
}

size_t smem_of(const fr_ctx* c, int kernel, int epb);

// threads per element of the element kernels, and the most elements a block
// may hold (1024 threads; at 64 threads per element, 15 named barriers)
int tpe_of(const fr_ctx* c) {
    if (c->prec == FR_FP64)
        return c->dim == 2 ? frl::threads_per_element<double, 2>(c->p) : frl::threads_per_element<double, 3>(c->p);
    return c->dim == 2 ? frl::threads_per_element<float, 2>(c->p) : frl::threads_per_element<float, 3>(c->p);
}
int max_epb(const fr_ctx* c) { return tpe_of(c) == 64 ? 15 : 32; }

// default: 8 warps (elements) per block, fewer when a block would need more
// than 96 KB of shared memory
void default_launch(fr_ctx* c) {
    for (int k = 0; k < 3; ++k) {
        int epb = 8;
        while (epb > 1 && smem_of(c, k, epb) > 96 * 1024) epb /= 2;
        c->lc[k].epb = epb;
        c->lc[k].threads = tpe_of(c) * epb;
    }
}

size_t smem_of(const fr_ctx* c, int kernel, int epb) {
    const bool cv = !c->affine;
    if (c->prec == FR_FP64)
        return c->dim == 2 ? frl::smem_bytes<double, 2>(c->p, kernel, epb, cv)
                           : frl::smem_bytes<double, 3>(c->p, kernel, epb, cv);
    return c->dim == 2 ? frl::smem_bytes<float, 2>(c->p, kernel, epb, cv) : frl::smem_bytes<float, 3>(c->p, kernel, epb, cv);
}

void release(fr_ctx* c) {
    if (!c) return;
    void* bufs[] = {c->u0, c->us, c->acc, c->ufb[0], c->ufb[1], c->fvn, c->S, c->J, c->iJ, c->N, c->nbr,
                    c->wall_ef, c->wall_off_d, c->fnow, c->fsum, c->fcnt, c->partial, c->stage64, c->dte,
                    c->fpart, c->src_elem, c->src_cand, c->src_w, c->src_A, c->src_f, c->tnow, c->dtc,
                    c->hlen, c->cand_off_d, c->lam, c->sp_elem, c->sp_cap, c->nonfinite, c->ufb3};
    for (void* b : bufs)
        if (b) cudaFree(b);
    for (int q = 0; q < frk::MAXNP; ++q) {
        void* rb[] = {c->red_elem[q], c->red_S[q], c->red_iJ[q]};
        for (void* b : rb)
            if (b) cudaFree(b);
    }
    if (c->order_d) cudaFree(c->order_d);
    for (auto& s : c->surf) {
        void* sb[] = {s.pe, s.pw, s.hist, s.count};
        for (void* b : sb)
            if (b) cudaFree(b);
    }
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (int q = 0; q < frk::MAXNP; ++q) {
        if (c->red_stream[q]) cudaStreamDestroy(c->red_stream[q]);
        if (c->ev_join[q]) cudaEventDestroy(c->ev_join[q]);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    delete c;
}

void invalidate_graph(fr_ctx* c) {
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
}

}  // namespace

// =====================================================================
int fr_set_error_from_fwh(int code, const char* msg) { return fail(code, msg); }

extern "C" const char* fr_last_error(void) { return g_err.c_str(); }

extern "C" int fr_ctx_dims(const fr_ctx* c, int64_t out[8]) {
    if (!c || !out) return fail(FR_EINVAL, "null argument");
    out[0] = c->dim;
    out[1] = c->p;
    out[2] = c->nv;
    out[3] = c->nsp;
    out[4] = c->E;
    out[5] = c->ncand;
    out[6] = c->prec;
    out[7] = c->affine + c->diag;
    return FR_OK;
}

extern "C" int fr_mesh_load(const fr_mesh_desc* m, int ncand, const fr_options* o, fr_ctx** out) {
    if (out) *out = nullptr;
    if (!m || !o || !out || ncand < 1) return fail(FR_EINVAL, "null argument or ncand < 1");
    const int dim = m[0].dim;
    if (dim != 2 && dim != 3) return fail(FR_EINVAL, "dim must be 2 or 3");
    if (o->order < 1 || o->order > 4) return fail(FR_EINVAL, "order must be 1..4");
    if (o->precision < FR_FP64 || o->precision > FR_BF16X3_TC) return fail(FR_EINVAL, "bad precision");
    if (o->precision >= FR_TF32_TC && (dim != 3 || o->order < 3))
        return fail(FR_EINVAL, "the tensor-core precision modes are built for 3D at p = 3 and 4");
    if (o->correction != FR_CORR_DG && o->correction != FR_CORR_HUYNH_G2) return fail(FR_EINVAL, "bad correction");
    if (!(o->gamma > 1.0) || !(o->prandtl > 0.0) || o->mu < 0.0 || !(o->rho_inf > 0.0) || !(o->p_inf > 0.0))
        return fail(FR_EINVAL, "bad gas or free-stream constants");
    if (o->viscous && !(o->mu > 0.0)) return fail(FR_EINVAL, "viscous run needs mu > 0");
    for (int c = 0; c < ncand; ++c) {
        if (m[c].dim != dim) return fail(FR_EINVAL, "all candidates must share dim");
        if (m[c].nelem < 1 || !m[c].nodes || !m[c].conn) return fail(FR_EINVAL, "empty mesh");
        if (m[c].geom_order != 1 && m[c].geom_order != 2) return fail(FR_EINVAL, "geom_order must be 1 or 2");
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1)
        return fail(FR_ECUDA, "no CUDA device available (libfr has no CPU path)");

    fr_ctx* c = new fr_ctx();
    cudaGetDevice(&c->device);
    c->dim = dim;
    c->p = o->order;
    c->np = c->p + 1;
    c->nsp = dim == 2 ? c->np * c->np : c->np * c->np * c->np;
    c->nfp = dim == 2 ? c->np : c->np * c->np;
    c->nf = 2 * dim;
    c->nv = dim + 2;
    c->ncand = ncand;
    c->prec = o->precision;
    c->visc = o->viscous ? 1 : 0;
    c->kind = o->correction;
    c->opt = *o;
    if (c->opt.br2_eta == 0.0) c->opt.br2_eta = 1.0;
    c->rsz = c->prec == FR_FP64 ? 8 : 4;
    frg::build_ref(c->p, c->kind, c->ref);
    c->cand_off.assign(ncand + 1, 0);
    for (int k = 0; k < ncand; ++k) c->cand_off[k + 1] = c->cand_off[k] + m[k].nelem;
    const int64_t E = c->E = c->cand_off[ncand];
    const int nsp = c->nsp, nfp = c->nfp, nf = c->nf, nv = c->nv;
    c->nodes.resize(ncand);
    c->q.resize(ncand);
    for (int k = 0; k < ncand; ++k) {
        const int nq = m[k].geom_order + 1;
        const int nn = dim == 2 ? nq * nq : nq * nq * nq;
        c->q[k] = m[k].geom_order;
        c->nodes[k].assign(m[k].nodes, m[k].nodes + int64_t(m[k].nelem) * nn * dim);
    }

    // ---- geometry (host, double), parallel over elements
    std::vector<double> Jh(E * nsp), Sh(E * dim * dim * nsp), Nown(E * nf * nfp * dim);
    std::vector<int> bad(1, 0);
    {
        unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
        std::vector<std::thread> th;
        std::vector<int> badj(nth, 0);
        for (unsigned t = 0; t < nth; ++t)
            th.emplace_back([&, t]() {
                std::vector<double> xsp(nsp * dim);
                for (int64_t e = t; e < E; e += nth) {
                    int k = int(std::upper_bound(c->cand_off.begin(), c->cand_off.end(), e) - c->cand_off.begin()) - 1;
                    const int q = c->q[k];
                    const int nq = q + 1;
                    const int nn = dim == 2 ? nq * nq : nq * nq * nq;
                    const double* nd = c->nodes[k].data() + (e - c->cand_off[k]) * nn * dim;
                    frg::element_geometry(dim, q, c->ref, nd, xsp.data(), &Jh[e * nsp], &Sh[e * dim * dim * nsp],
                                          &Nown[e * nf * nfp * dim]);
                    for (int s = 0; s < nsp; ++s)
                        if (!(Jh[e * nsp + s] > 0.0)) badj[t] = 1;
                }
            });
        for (auto& x : th) x.join();
        for (int b : badj) bad[0] |= b;
    }
    if (bad[0]) {
        release(c);
        return fail(FR_EMESH, "non-positive Jacobian at a solution point");
    }

    // ---- connectivity, shared normals
    std::vector<int32_t> nbr(E * nf);
    std::vector<double> Nsh(Nown);
    std::vector<std::vector<int32_t>> walls(ncand);
    for (int k = 0; k < ncand; ++k) {
        const int64_t off = c->cand_off[k];
        const int ne = m[k].nelem;
        const int32_t* cn = m[k].conn;
        for (int e = 0; e < ne; ++e)
            for (int f = 0; f < nf; ++f) {
                const int32_t a = cn[(int64_t(e) * nf + f) * 3 + 0];
                const int32_t b = cn[(int64_t(e) * nf + f) * 3 + 1];
                const int32_t oc = cn[(int64_t(e) * nf + f) * 3 + 2];
                const int64_t ge = off + e;
                if (a < 0) {
                    if (a != -FR_BC_WALL && a != -FR_BC_FARFIELD) {
                        release(c);
                        return fail(FR_EMESH, "unknown boundary tag");
                    }
                    nbr[ge * nf + f] = a;
                    if (a == -FR_BC_WALL) walls[k].push_back(int32_t(ge * nf + f));
                    continue;
                }
                if (a >= ne || b < 0 || b >= nf || oc < 0 || oc >= (dim == 2 ? 2 : 8)) {
                    release(c);
                    return fail(FR_EMESH, "connectivity entry out of range");
                }
                const int32_t* back = cn + (int64_t(a) * nf + b) * 3;
                if (back[0] != e || back[1] != f) {
                    release(c);
                    return fail(FR_EMESH, "connectivity is not symmetric");
                }
                for (int fp = 0; fp < nfp; ++fp)
                    if (orient_map(dim, c->np, back[2], orient_map(dim, c->np, oc, fp)) != fp) {
                        release(c);
                        return fail(FR_EMESH, "face orientations are not inverse to each other");
                    }
                const int64_t gn = off + a;
                if ((gn * nf + b) * 8 + oc > INT32_MAX) {
                    release(c);
                    return fail(FR_EINVAL, "mesh too large for 32-bit face codes");
                }
                nbr[ge * nf + f] = int32_t((gn * nf + b) * 8 + oc);
                // normals: both sides must agree (opposite) -- a mismatch means
                // the connectivity pairs faces that do not coincide
                double nmax = 0.0, dmax = 0.0;
                for (int fp = 0; fp < nfp; ++fp) {
                    const int fq = orient_map(dim, c->np, oc, fp);
                    for (int i = 0; i < dim; ++i) {
                        const double x = Nown[((ge * nf + f) * nfp + fp) * dim + i];
                        const double y = Nown[((gn * nf + b) * nfp + fq) * dim + i];
                        nmax = std::max(nmax, std::fabs(x));
                        dmax = std::max(dmax, std::fabs(x + y));
                    }
                }
                if (dmax > 1e-6 * nmax + 1e-300) {
                    release(c);
                    return fail(FR_EMESH, "matched faces have inconsistent normals (wrong connectivity or orientation)");
                }
                if (ge * nf + f > gn * nf + b)
                    for (int fp = 0; fp < nfp; ++fp) {
                        const int fq = orient_map(dim, c->np, oc, fp);
                        for (int i = 0; i < dim; ++i)
                            Nsh[((ge * nf + f) * nfp + fp) * dim + i] = -Nown[((gn * nf + b) * nfp + fq) * dim + i];
                    }
            }
    }

    // ---- affine detection: constant metrics per element and normals per face.
    // Each metric row S[d][:] (the area vector of the xi_d faces) and each
    // face normal is compared against its own largest component, so round-off
    // in components that vanish analytically (axis-aligned elements) does not
    // count as variation.
    bool affine = true;
    for (int64_t e = 0; e < E && affine; ++e) {
        for (int d = 0; d < dim && affine; ++d) {
            double mx = 0;
            for (int i = 0; i < dim; ++i)
                for (int sp = 0; sp < nsp; ++sp) mx = std::max(mx, std::fabs(Sh[(e * dim * dim + d * dim + i) * nsp + sp]));
            for (int i = 0; i < dim && affine; ++i) {
                const double* s = &Sh[(e * dim * dim + d * dim + i) * nsp];
                for (int sp = 1; sp < nsp; ++sp)
                    if (std::fabs(s[sp] - s[0]) > 1e-13 * mx) affine = false;
            }
        }
        for (int sp = 1; sp < nsp && affine; ++sp)
            if (std::fabs(Jh[e * nsp + sp] - Jh[e * nsp]) > 1e-13 * std::fabs(Jh[e * nsp])) affine = false;
        for (int f = 0; f < nf && affine; ++f) {
            const double* nv = &Nsh[(e * nf + f) * nfp * dim];
            double mx = 0;
            for (int k = 0; k < nfp * dim; ++k) mx = std::max(mx, std::fabs(nv[k]));
            for (int fp = 1; fp < nfp && affine; ++fp)
                for (int i = 0; i < dim; ++i)
                    if (std::fabs(nv[fp * dim + i] - nv[i]) > 1e-13 * mx) affine = false;
        }
    }
    c->affine = affine ? 1 : 0;
    // element length of the adaptive time step: min over points and
    // directions of 2 |J| / |S[d,:]|
    std::vector<double> hl(size_t(E), 1e300);
    for (int64_t e = 0; e < E; ++e)
        for (int d = 0; d < dim; ++d)
            for (int sp = 0; sp < nsp; ++sp) {
                double n2 = 0.0;
                for (int i = 0; i < dim; ++i) {
                    const double v = Sh[(e * dim * dim + d * dim + i) * nsp + sp];
                    n2 += v * v;
                }
                hl[e] = std::min(hl[e], 2.0 * Jh[e * nsp + sp] / std::sqrt(n2));
            }
    int rc;
    if ((rc = upload_real(&c->hlen, hl, c->prec)) ||
        (rc = upload(reinterpret_cast<void**>(&c->cand_off_d), c->cand_off))) {
        release(c);
        return rc;
    }
    if (affine) {
        std::vector<double> S1(E * dim * dim), J1(E), N1(E * nf * dim);
        for (int64_t e = 0; e < E; ++e) {
            for (int k = 0; k < dim * dim; ++k) S1[e * dim * dim + k] = Sh[(e * dim * dim + k) * nsp];
            J1[e] = Jh[e * nsp];
            for (int f = 0; f < nf; ++f)
                for (int i = 0; i < dim; ++i) N1[(e * nf + f) * dim + i] = Nsh[((e * nf + f) * nfp) * dim + i];
        }
        // axis-aligned elements: when every off-diagonal S entry of every
        // element is round-off (at most 1e-13 of its row's largest entry),
        // those entries become exact zeros and the kernels skip them
        bool diag = true;
        for (int64_t e = 0; e < E && diag; ++e)
            for (int d = 0; d < dim && diag; ++d) {
                const double* row = &S1[e * dim * dim + d * dim];
                double mx = 0.0;
                for (int i = 0; i < dim; ++i) mx = std::max(mx, std::fabs(row[i]));
                for (int i = 0; i < dim; ++i)
                    if (i != d && std::fabs(row[i]) > 1e-13 * mx) diag = false;
            }
        for (int64_t e = 0; e < E && diag; ++e)
            for (int f = 0; f < nf && diag; ++f) {
                const double* nv = &N1[(e * nf + f) * dim];
                double mx = 0.0;
                for (int i = 0; i < dim; ++i) mx = std::max(mx, std::fabs(nv[i]));
                for (int i = 0; i < dim; ++i)
                    if (i != f / 2 && std::fabs(nv[i]) > 1e-13 * mx) diag = false;
            }
        // (and so do the matching components of the face normals: the normal of
        // a face of direction d lies along axis d, which the kernels assume)
        if (diag)
            for (int64_t e = 0; e < E; ++e) {
                for (int d = 0; d < dim; ++d)
                    for (int i = 0; i < dim; ++i)
                        if (i != d) S1[e * dim * dim + d * dim + i] = 0.0;
                for (int f = 0; f < nf; ++f)
                    for (int i = 0; i < dim; ++i)
                        if (i != f / 2) N1[(e * nf + f) * dim + i] = 0.0;
            }
        c->diag = diag ? 1 : 0;
        // the larger (element, face) side takes the exact negative of the
        // smaller side's constant normal, so common fluxes stay equal and opposite
        for (int64_t e = 0; e < E; ++e)
            for (int f = 0; f < nf; ++f) {
                const int32_t code = nbr[e * nf + f];
                if (code < 0) continue;
                const int64_t other = code >> 3;
                if (e * nf + f > other)
                    for (int i = 0; i < dim; ++i) N1[(e * nf + f) * dim + i] = -N1[other * dim + i];
            }
        c->sS_e = dim * dim; c->sS_k = 1; c->sS_sp = 0;
        c->sJ_e = 1; c->sJ_sp = 0;
        c->sN_f = dim; c->sN_fp = 0;
        std::vector<double> iJ1(J1.size());
        for (size_t i = 0; i < J1.size(); ++i) iJ1[i] = 1.0 / J1[i];
        if ((rc = upload_real(&c->S, S1, c->prec)) || (rc = upload_real(&c->J, J1, c->prec)) ||
            (rc = upload_real(&c->iJ, iJ1, c->prec)) || (rc = upload_real(&c->N, N1, c->prec))) {
            release(c);
            return rc;
        }
    } else {
        c->sS_e = int64_t(dim) * dim * nsp; c->sS_k = nsp; c->sS_sp = 1;
        c->sJ_e = nsp; c->sJ_sp = 1;
        c->sN_f = int64_t(nfp) * dim; c->sN_fp = dim;
        std::vector<double> iJh(Jh.size());
        for (size_t i = 0; i < Jh.size(); ++i) iJh[i] = 1.0 / Jh[i];
        if ((rc = upload_real(&c->S, Sh, c->prec)) || (rc = upload_real(&c->J, Jh, c->prec)) ||
            (rc = upload_real(&c->iJ, iJh, c->prec)) || (rc = upload_real(&c->N, Nsh, c->prec))) {
            release(c);
            return rc;
        }
    }
    c->bnd = 0;
    for (const int32_t code : nbr)
        if (code < 0) c->bnd = 1;
    if ((rc = upload(reinterpret_cast<void**>(&c->nbr), nbr))) {
        release(c);
        return rc;
    }
    // walls per candidate
    std::vector<int32_t> wl;
    c->wall_off.assign(ncand + 1, 0);
    for (int k = 0; k < ncand; ++k) {
        wl.insert(wl.end(), walls[k].begin(), walls[k].end());
        c->wall_off[k + 1] = int64_t(wl.size());
    }
    if ((rc = upload(reinterpret_cast<void**>(&c->wall_ef), wl)) ||
        (rc = upload(reinterpret_cast<void**>(&c->wall_off_d), c->wall_off))) {
        release(c);
        return rc;
    }
    // operators (passed to kernels by value)
    c->opd = ops_of<double>(c->ref);
    c->opf = ops_of<float>(c->ref);
    // state and trace buffers
    const size_t nstate = size_t(E) * nv * nsp * c->rsz;
    const size_t ntrace = size_t(E) * nf * nv * nfp * c->rsz;
    if (cudaMalloc(&c->u0, nstate) != cudaSuccess || cudaMalloc(&c->us, nstate) != cudaSuccess ||
        cudaMalloc(&c->acc, nstate) != cudaSuccess || cudaMalloc(&c->ufb[0], ntrace) != cudaSuccess ||
        cudaMalloc(&c->ufb[1], ntrace) != cudaSuccess || cudaMalloc(&c->fvn, ntrace) != cudaSuccess) {
        release(c);
        return fail(FR_ENOMEM, "cudaMalloc failed for the state buffers");
    }
    cudaMemset(c->u0, 0, nstate);
    cudaMemset(c->us, 0, nstate);
    cudaMemset(c->acc, 0, nstate);
    cudaMemset(c->ufb[0], 0, ntrace);
    cudaMemset(c->ufb[1], 0, ntrace);
    cudaMemset(c->fvn, 0, ntrace);
    c->partial_blocks = 1024;
    if (cudaMalloc(&c->fnow, sizeof(double) * 3 * ncand) != cudaSuccess ||
        cudaMalloc(&c->fsum, sizeof(double) * 3 * ncand) != cudaSuccess ||
        cudaMalloc(&c->fcnt, sizeof(double) * ncand) != cudaSuccess ||
        cudaMalloc(&c->partial, sizeof(double) * c->partial_blocks * (nv + 1)) != cudaSuccess ||
        cudaMalloc(&c->fpart, sizeof(double) * 3 * frk::FORCE_BLOCKS * ncand) != cudaSuccess) {
        release(c);
        return fail(FR_ENOMEM, "cudaMalloc failed for accumulators");
    }
    cudaMemset(c->fnow, 0, sizeof(double) * 3 * ncand);
    cudaMemset(c->fsum, 0, sizeof(double) * 3 * ncand);
    cudaMemset(c->fcnt, 0, sizeof(double) * ncand);
    if (cudaMalloc(&c->nonfinite, sizeof(int) * ncand) != cudaSuccess) {
        c->nonfinite = nullptr;
        release(c);
        return fail(FR_ENOMEM, "cudaMalloc failed for the non-finite flags");
    }
    cudaMemset(c->nonfinite, 0, sizeof(int) * ncand);
    bool streams_ok = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) == cudaSuccess &&
                      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int q = 0; q < c->p && streams_ok; ++q)
        streams_ok = cudaStreamCreateWithFlags(&c->red_stream[q], cudaStreamNonBlocking) == cudaSuccess &&
                     cudaEventCreateWithFlags(&c->ev_join[q], cudaEventDisableTiming) == cudaSuccess;
    if (!streams_ok) {
        release(c);
        return fail(FR_ECUDA, "cannot create a stream");
    }
    default_launch(c);
    c->cand_dt.assign(ncand, o->dt);
    c->srcs.assign(ncand, {});
    {
        // first use of each kernel: shared-memory opt-in outside any capture
        const int64_t keepE = c->E;
        c->E = 0;
        int r0, r1, r2;
        if (c->prec == FR_FP64) {
            frk::Stage<double> st{0, 0.0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
            r0 = L_traces<double>(c, nullptr, nullptr, nullptr);
            r1 = L_visc<double>(c, nullptr, nullptr, nullptr);
            r2 = L_resid<double>(c, nullptr, nullptr, st, nullptr);
        } else {
            frk::Stage<float> st{0, 0.0f, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
            r0 = L_traces<float>(c, nullptr, nullptr, nullptr);
            r1 = L_visc<float>(c, nullptr, nullptr, nullptr);
            r2 = L_resid<float>(c, nullptr, nullptr, st, nullptr);
        }
        c->E = keepE;
        c->launches = 0;
        if (r0 || r1 || r2) {
            release(c);
            return fail(FR_ECUDA, std::string("kernel set-up: ") + cudaGetErrorString(cudaError_t(r0 | r1 | r2)));
        }
    }
    cudaError_t err = cudaDeviceSynchronize();
    if (err != cudaSuccess) {
        release(c);
        return fail(FR_ECUDA, std::string("set-up: ") + cudaGetErrorString(err));
    }
    *out = c;
    return FR_OK;
}

extern "C" int fr_destroy(fr_ctx* c) {
    if (!c) return FR_OK;
    cudaDeviceSynchronize();
    release(c);
    return FR_OK;
}

extern "C" int fr_cand_range(const fr_ctx* c, int cand, int64_t* first, int64_t* count) {
    if (!c || !first || !count) return fail(FR_EINVAL, "null argument");
    if (cand < 0) {
        *first = 0;
        *count = c->E;
        return FR_OK;
    }
    if (cand >= c->ncand) return fail(FR_EINVAL, "candidate out of range");
    *first = c->cand_off[cand];
    *count = c->cand_off[cand + 1] - c->cand_off[cand];
    return FR_OK;
}

extern "C" int fr_sp_coords(const fr_ctx* c, int cand, double* xyz) {
    if (!c || !xyz) return fail(FR_EINVAL, "null argument");
    int64_t first, count;
    int rc = fr_cand_range(c, cand, &first, &count);
    if (rc) return rc;
    const int dim = c->dim, nsp = c->nsp, nf = c->nf, nfp = c->nfp;
    std::vector<double> J(nsp), S(dim * dim * nsp), N(nf * nfp * dim);
    for (int64_t e = first; e < first + count; ++e) {
        int k = int(std::upper_bound(c->cand_off.begin(), c->cand_off.end(), e) - c->cand_off.begin()) - 1;
        const int nq = c->q[k] + 1;
        const int nn = dim == 2 ? nq * nq : nq * nq * nq;
        frg::element_geometry(dim, c->q[k], c->ref, c->nodes[k].data() + (e - c->cand_off[k]) * nn * dim,
                              xyz + (e - first) * nsp * dim, J.data(), S.data(), N.data());
    }
    return FR_OK;
}

extern "C" int fr_state_set(fr_ctx* c, int cand, const double* u, int on_device, void* stream) {
    if (!c || !u) return fail(FR_EINVAL, "null argument");
    int64_t first, count;
    int rc = fr_cand_range(c, cand, &first, &count);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = count * c->nv * c->nsp;
    char* dst = static_cast<char*>(c->u0) + first * c->nv * c->nsp * c->rsz;
    c->traces_valid = false;
    CK(cudaMemsetAsync(c->nonfinite + (cand < 0 ? 0 : cand), 0, sizeof(int) * (cand < 0 ? c->ncand : 1), s));
    const double* hu = on_device ? nullptr : static_cast<const double*>(host_alias(u));
    if (c->prec == FR_FP64 && hu) {
        k_d2d<<<2048, 256, 0, s>>>(hu, reinterpret_cast<double*>(dst), n);
        ++c->launches;
        CK(cudaGetLastError());
    } else if (c->prec == FR_FP64) {
        CK(cudaMemcpyAsync(dst, u, n * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    } else if (on_device || hu) {
        k_d2f<<<2048, 256, 0, s>>>(on_device ? u : hu, reinterpret_cast<float*>(dst), n);
        ++c->launches;
        CK(cudaGetLastError());
    } else {
        // host doubles -> device staging -> float on the device
        if (!c->stage64 && cudaMalloc(&c->stage64, size_t(c->E) * c->nv * c->nsp * 8) != cudaSuccess) {
            c->stage64 = nullptr;
            return fail(FR_ENOMEM, "cannot allocate the transfer staging buffer");
        }
        CK(cudaMemcpyAsync(c->stage64, u, n * 8, cudaMemcpyHostToDevice, s));
        k_d2f<<<1024, 256, 0, s>>>(c->stage64, reinterpret_cast<float*>(dst), n);
        ++c->launches;
        CK(cudaGetLastError());
    }
    if (c->sp_n > 0) {
        rc = c->prec == FR_FP64 ? L_sponge<double>(c, static_cast<double*>(c->u0), nullptr, nullptr, s, cand)
                                : L_sponge<float>(c, static_cast<float*>(c->u0), nullptr, nullptr, s, cand);
        CKL(rc, "sponge kernel");
    }
    CK(cudaStreamSynchronize(s));
    return FR_OK;
}

extern "C" int fr_state_get(fr_ctx* c, int cand, double* u, int on_device, void* stream) {
    if (!c || !u) return fail(FR_EINVAL, "null argument");
    int64_t first, count;
    int rc = fr_cand_range(c, cand, &first, &count);
    if (rc) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t n = count * c->nv * c->nsp;
    const char* src = static_cast<const char*>(c->u0) + first * c->nv * c->nsp * c->rsz;
    double* hu = on_device ? nullptr : static_cast<double*>(const_cast<void*>(host_alias(u)));
    if (c->prec == FR_FP64 && hu) {
        k_d2d<<<2048, 256, 0, s>>>(reinterpret_cast<const double*>(src), hu, n);
        ++c->launches;
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s));
    } else if (c->prec == FR_FP64) {
        CK(cudaMemcpyAsync(u, src, n * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } else if (on_device || hu) {
        k_f2d<<<2048, 256, 0, s>>>(reinterpret_cast<const float*>(src), on_device ? u : hu, n);
        ++c->launches;
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s));
    } else {
        if (!c->stage64 && cudaMalloc(&c->stage64, size_t(c->E) * c->nv * c->nsp * 8) != cudaSuccess) {
            c->stage64 = nullptr;
            return fail(FR_ENOMEM, "cannot allocate the transfer staging buffer");
        }
        k_f2d<<<1024, 256, 0, s>>>(reinterpret_cast<const float*>(src), c->stage64, n);
        ++c->launches;
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(u, c->stage64, n * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    if (!on_device) {
        for (int64_t i = 0; i < n; ++i)
            if (!std::isfinite(u[i])) return fail(FR_ENONFINITE, "state holds NaN or Inf");
    }
    // flags set on the device by the last stage of a step
    for (int k = (cand < 0 ? 0 : cand); k < (cand < 0 ? c->ncand : cand + 1); ++k) {
        int bad = 0;
        CK(cudaMemcpy(&bad, c->nonfinite + k, sizeof(int), cudaMemcpyDeviceToHost));
        if (bad) return fail(FR_ENONFINITE, "candidate " + std::to_string(k) + ": a step produced NaN or Inf");
    }
    return FR_OK;
}

extern "C" int fr_nonfinite(const fr_ctx* c, int cand, int* flag) {
    if (!c || !flag || cand < -1 || cand >= c->ncand) return fail(FR_EINVAL, "bad argument");
    CK(cudaDeviceSynchronize());
    *flag = 0;
    for (int k = (cand < 0 ? 0 : cand); k < (cand < 0 ? c->ncand : cand + 1); ++k) {
        int bad = 0;
        CK(cudaMemcpy(&bad, c->nonfinite + k, sizeof(int), cudaMemcpyDeviceToHost));
        *flag |= bad ? 1 : 0;
    }
    return FR_OK;
}

extern "C" int fr_set_rk_scheme(fr_ctx* c, int nstages, const double* coef) {
    if (!c || nstages < 0 || nstages > 16 || (nstages > 0 && !coef)) return fail(FR_EINVAL, "bad argument");
    if (nstages == 0) {
        c->lsc.clear();
        c->ls_time.clear();
        invalidate_graph(c);
        return FR_OK;
    }
    std::vector<std::array<double, 6>> k(nstages);
    for (int i = 0; i < nstages; ++i)
        for (int j = 0; j < 6; ++j) {
            k[i][j] = coef[i * 6 + j];
            if (!std::isfinite(k[i][j])) return fail(FR_EINVAL, "non-finite scheme coefficient");
        }
    // stage abscissae from the scheme applied to du/dt = 1 (u = t, dt = 1):
    // the value of each stage's input is its time; one step must reach 1
    std::vector<double> tin(nstages);
    double v = 0.0, acc = 0.0;
    for (int i = 0; i < nstages; ++i) {
        tin[i] = v;
        acc = (i == 0 ? 0.0 : k[i][4] * acc) + k[i][5];
        v = k[i][0] * 0.0 + k[i][1] * v + k[i][2] + k[i][3] * acc;
    }
    if (!(std::fabs(v - 1.0) <= 1e-12))
        return fail(FR_EINVAL, "inconsistent scheme: one step of du/dt = 1 must advance u by dt");
    if (nstages % 2 == 1 && nstages > 1 && !c->ufb3) {
        const size_t ntrace = size_t(c->E) * c->nf * c->nv * c->nfp * c->rsz;
        if (cudaMalloc(&c->ufb3, ntrace) != cudaSuccess) {
            c->ufb3 = nullptr;
            return fail(FR_ENOMEM, "cannot allocate the third trace buffer");
        }
    }
    c->lsc = k;
    c->ls_time = tin;
    invalidate_graph(c);
    return FR_OK;
}

extern "C" int fr_residual(fr_ctx* c, const void* u, void* R, void* stream) {
    if (!c || !u || !R) return fail(FR_EINVAL, "null argument");
    if (u == R) return fail(FR_EINVAL, "u and R must not overlap");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (c->prec == FR_FP64)
        return enqueue_residual<double>(c, static_cast<const double*>(u), static_cast<double*>(R), s);
    return enqueue_residual<float>(c, static_cast<const float*>(u), static_cast<float*>(R), s);
}

extern "C" int fr_rk_step(fr_ctx* c, int nsteps, void* stream) {
    if (!c || nsteps < 0) return fail(FR_EINVAL, "bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = c->prec == FR_FP64 ? ensure_traces<double>(c, s) : ensure_traces<float>(c, s);
    if (rc) return rc;
    for (int k = 0; k < nsteps; ++k) {
        rc = c->prec == FR_FP64 ? enqueue_step<double>(c, s) : enqueue_step<float>(c, s);
        if (rc) return rc;
    }
    return FR_OK;
}

extern "C" int fr_rk_step_graph(fr_ctx* c, int nsteps, void* stream) {
    if (!c || nsteps < 0) return fail(FR_EINVAL, "bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        const int rc = c->prec == FR_FP64 ? ensure_traces<double>(c, s) : ensure_traces<float>(c, s);
        if (rc) return rc;
    }
    if (!c->gexec) {
        // make sure every kernel attribute is set before capture
        CK(cudaStreamSynchronize(s));
        const int64_t before = c->launches;
        CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        const int rc = c->prec == FR_FP64 ? enqueue_step<double>(c, c->cap_stream)
                                          : enqueue_step<float>(c, c->cap_stream);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(c->cap_stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (ec != cudaSuccess) return fail(FR_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
        const cudaError_t ei = cudaGraphInstantiate(&c->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            c->gexec = nullptr;
            return fail(FR_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
        }
        c->graph_launches_per_step = c->launches - before;
        c->launches = before;
    }
    for (int k = 0; k < nsteps; ++k) {
        CK(cudaGraphLaunch(c->gexec, s));
        c->launches += c->graph_launches_per_step;
    }
    return FR_OK;
}

__global__ void k_fill_d(double* a, int64_t n, double v) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        a[i] = v;
}
__global__ void k_fill_f(float* a, int64_t n, float v) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        a[i] = v;
}

extern "C" int fr_set_cand_dt(fr_ctx* c, int cand, double dt) {
    if (!c || cand < 0 || cand >= c->ncand || !(dt > 0.0)) return fail(FR_EINVAL, "bad candidate or dt");
    CK(cudaDeviceSynchronize());
    c->cand_dt[cand] = dt;
    if (c->dtc) CK(cudaMemcpy(c->dtc + cand, &dt, sizeof(double), cudaMemcpyHostToDevice));
    if (!c->dte) {
        if (cudaMalloc(&c->dte, size_t(c->E) * c->rsz) != cudaSuccess) {
            c->dte = nullptr;
            return fail(FR_ENOMEM, "cannot allocate per-element time steps");
        }
        if (c->prec == FR_FP64) k_fill_d<<<256, 256>>>(static_cast<double*>(c->dte), c->E, c->opt.dt);
        else k_fill_f<<<256, 256>>>(static_cast<float*>(c->dte), c->E, float(c->opt.dt));
        c->launches += 1;
        CK(cudaGetLastError());
        invalidate_graph(c);  // the captured step read the scalar dt
    }
    const int64_t a0 = c->cand_off[cand], n = c->cand_off[cand + 1] - a0;
    if (c->prec == FR_FP64) k_fill_d<<<256, 256>>>(static_cast<double*>(c->dte) + a0, n, dt);
    else k_fill_f<<<256, 256>>>(static_cast<float*>(c->dte) + a0, n, float(dt));
    c->launches += 1;
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    return FR_OK;
}

// ---------------------------------------------------------------- energy sources (Appendix D)
namespace {

template <typename Real>
int upload_src_weights(fr_ctx* c, const std::vector<double>& w) {
    std::vector<Real> h(w.begin(), w.end());
    if (cudaMalloc(&c->src_w, sizeof(Real) * std::max<size_t>(1, h.size())) != cudaSuccess) return FR_ENOMEM;
    if (!h.empty() && cudaMemcpy(c->src_w, h.data(), sizeof(Real) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return FR_ECUDA;
    return FR_OK;
}

// Rebuilds the device source table from c->srcs: every element with a
// solution point where some exp(-k_m |x - x_m|^2) exceeds 1e-30 gets an entry.
int rebuild_sources(fr_ctx* c) {
    for (void** b : {reinterpret_cast<void**>(&c->src_elem), reinterpret_cast<void**>(&c->src_cand), &c->src_w}) {
        if (*b) cudaFree(*b);
        *b = nullptr;
    }
    c->src_nentry = 0;
    bool any = false;
    for (const auto& v : c->srcs) any = any || !v.empty();
    if (!any) return FR_OK;
    const int dim = c->dim, nsp = c->nsp, nf = c->nf, nfp = c->nfp, M = frk::MAXSRC;
    std::vector<int32_t> elem_of, cand_of;
    std::vector<double> w;
    std::vector<double> xyz(size_t(nsp) * dim), J(nsp), S(size_t(dim) * dim * nsp), N(size_t(nf) * nfp * dim);
    for (int k = 0; k < c->ncand; ++k) {
        const auto& sv = c->srcs[k];
        if (sv.empty()) continue;
        const int nq = c->q[k] + 1;
        const int nn = dim == 2 ? nq * nq : nq * nq * nq;
        for (int64_t e = c->cand_off[k]; e < c->cand_off[k + 1]; ++e) {
            frg::element_geometry(dim, c->q[k], c->ref, c->nodes[k].data() + (e - c->cand_off[k]) * nn * dim,
                                  xyz.data(), J.data(), S.data(), N.data());
            std::vector<double> we(size_t(M) * nsp, 0.0);
            bool active = false;
            for (size_t m = 0; m < sv.size(); ++m)
                for (int sp = 0; sp < nsp; ++sp) {
                    double r2 = 0.0;
                    for (int i = 0; i < dim; ++i) {
                        const double d = xyz[size_t(sp) * dim + i] - sv[m][2 + i];
                        r2 += d * d;
                    }
                    const double v = std::exp(-sv[m][1] * r2);
                    we[m * nsp + sp] = v;
                    if (v > 1e-30) active = true;
                }
            if (!active) continue;
            elem_of.push_back(int32_t(e));
            cand_of.push_back(k);
            w.insert(w.end(), we.begin(), we.end());
        }
    }
    std::vector<double> A(size_t(c->ncand) * M, 0.0), f(size_t(c->ncand) * M, 0.0);
    for (int k = 0; k < c->ncand; ++k)
        for (size_t m = 0; m < c->srcs[k].size(); ++m) {
            A[size_t(k) * M + m] = c->srcs[k][m][0];
            f[size_t(k) * M + m] = c->srcs[k][m][5];
        }
    int rc;
    if (cand_of.empty()) return FR_OK;   // sources too far from every solution point
    if ((rc = upload(reinterpret_cast<void**>(&c->src_elem), elem_of)) ||
        (rc = upload(reinterpret_cast<void**>(&c->src_cand), cand_of)))
        return rc;
    rc = c->prec == FR_FP64 ? upload_src_weights<double>(c, w) : upload_src_weights<float>(c, w);
    if (rc) return rc;
    if (cudaMemcpy(c->src_A, A.data(), A.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->src_f, f.data(), f.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
        return FR_ECUDA;
    c->src_nentry = int(cand_of.size());
    return FR_OK;
}

// host copy (as double) of n consecutive Reals of a device array
int download_real(const fr_ctx* c, const void* d, int64_t off, int64_t n, double* out) {
    if (n <= 0) return FR_OK;
    if (c->prec == FR_FP64) {
        if (cudaMemcpy(out, static_cast<const double*>(d) + off, size_t(n) * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
            return FR_ECUDA;
        return FR_OK;
    }
    std::vector<float> f(static_cast<size_t>(n));
    if (cudaMemcpy(f.data(), static_cast<const float*>(d) + off, size_t(n) * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return FR_ECUDA;
    for (int64_t i = 0; i < n; ++i) out[i] = f[size_t(i)];
    return FR_OK;
}

// in [np^dim] -> out [nq^dim]: M [nq][np] along every direction (direction 0 fastest)
void interp_vol(int dim, int np, int nq, const double* M, const double* in, double* out) {
    std::vector<double> a(in, in + (dim == 2 ? np * np : np * np * np)), b;
    int n[3] = {np, np, dim == 3 ? np : 1};
    for (int d = 0; d < dim; ++d) {
        int m[3] = {n[0], n[1], n[2]};
        m[d] = nq;
        b.assign(size_t(m[0]) * m[1] * m[2], 0.0);
        for (int i2 = 0; i2 < m[2]; ++i2)
            for (int i1 = 0; i1 < m[1]; ++i1)
                for (int i0 = 0; i0 < m[0]; ++i0) {
                    const int o[3] = {i0, i1, i2};
                    double acc = 0.0;
                    for (int j = 0; j < n[d]; ++j) {
                        int ii[3] = {i0, i1, i2};
                        ii[d] = j;
                        acc += M[o[d] * frk::MAXNP + j] * a[(size_t(ii[2]) * n[1] + ii[1]) * n[0] + ii[0]];
                    }
                    b[(size_t(i2) * m[1] + i1) * m[0] + i0] = acc;
                }
        a.swap(b);
        n[d] = nq;
    }
    std::copy(a.begin(), a.end(), out);
}

// The reduced-element tables of the kernels of frk::Red from c->order: per
// degree q < p the element list and the metric terms at the q points (the
// degree-p interpolants of S and |J| evaluated there, 1/|J| stored), and the
// per-element degrees.
int build_reduced(fr_ctx* c) {
    for (int q = 0; q < frk::MAXNP; ++q) {
        void* rb[] = {c->red_elem[q], c->red_S[q], c->red_iJ[q]};
        for (void* b : rb)
            if (b) cudaFree(b);
        c->red_elem[q] = nullptr;
        c->red_S[q] = c->red_iJ[q] = nullptr;
        c->red_n[q] = 0;
    }
    if (c->order_d) cudaFree(c->order_d);
    c->order_d = nullptr;
    const int dim = c->dim, np = c->np, nsp = c->nsp;
    std::vector<std::vector<int32_t>> lists(size_t(c->p));
    std::vector<signed char> ord(size_t(c->E), static_cast<signed char>(c->p));
    bool any = false;
    for (int k = 0; k < c->ncand; ++k)
        for (size_t i = 0; i < c->order[k].size(); ++i)
            if (c->order[k][i] < c->p) {
                const int64_t e = c->cand_off[k] + int64_t(i);
                lists[size_t(c->order[k][i])].push_back(int32_t(e));
                ord[size_t(e)] = static_cast<signed char>(c->order[k][i]);
                any = true;
            }
    if (!any) return FR_OK;
    int rc;
    if ((rc = upload(reinterpret_cast<void**>(&c->order_d), ord))) return rc;
    std::vector<double> Se(static_cast<size_t>(dim) * dim * nsp), Je(static_cast<size_t>(nsp)),
        tmp(static_cast<size_t>(dim) * dim + 1);
    for (int q = 0; q < c->p; ++q) {
        const auto& el = lists[size_t(q)];
        if (el.empty()) continue;
        const int nq = q + 1, nsq = dim == 2 ? nq * nq : nq * nq * nq;
        const auto rd = red_of<double>(c, q);
        std::vector<double> Sq(el.size() * size_t(dim) * dim * nsq), iJq(el.size() * size_t(nsq));
        for (size_t k = 0; k < el.size(); ++k) {
            const int64_t e = el[k];
            // S[e*sS_e + kk*sS_k + sp*sS_sp] and J[e*sJ_e + sp*sJ_sp] (stride 0: affine)
            if (c->sS_sp == 0) {
                if ((rc = download_real(c, c->S, e * c->sS_e, int64_t(dim) * dim, tmp.data()))) return rc;
                for (int kk = 0; kk < dim * dim; ++kk)
                    for (int sp = 0; sp < nsp; ++sp) Se[size_t(kk) * nsp + sp] = tmp[size_t(kk)];
            } else {
                if ((rc = download_real(c, c->S, e * c->sS_e, int64_t(dim) * dim * nsp, Se.data()))) return rc;
            }
            if (c->sJ_sp == 0) {
                if ((rc = download_real(c, c->J, e * c->sJ_e, 1, tmp.data()))) return rc;
                std::fill(Je.begin(), Je.end(), tmp[0]);
            } else {
                if ((rc = download_real(c, c->J, e * c->sJ_e, nsp, Je.data()))) return rc;
            }
            for (int kk = 0; kk < dim * dim; ++kk)
                interp_vol(dim, np, nq, rd.Iqp, Se.data() + size_t(kk) * nsp, Sq.data() + (k * dim * dim + kk) * nsq);
            interp_vol(dim, np, nq, rd.Iqp, Je.data(), iJq.data() + k * nsq);
            for (int pt = 0; pt < nsq; ++pt) iJq[k * nsq + pt] = 1.0 / iJq[k * nsq + pt];
        }
        if ((rc = upload(reinterpret_cast<void**>(&c->red_elem[q]), el)) ||
            (rc = upload_real(&c->red_S[q], Sq, c->prec)) || (rc = upload_real(&c->red_iJ[q], iJq, c->prec)))
            return rc;
        c->red_n[q] = int(el.size());
    }
    return FR_OK;
}

}  // namespace

extern "C" int fr_set_source(fr_ctx* c, int cand, int nsrc, const double* src, double t0) {
    if (!c || cand < 0 || cand >= c->ncand || nsrc < 0 || nsrc > frk::MAXSRC || (nsrc > 0 && !src) ||
        !std::isfinite(t0))
        return fail(FR_EINVAL, "bad argument (0 <= nsrc <= 4 sources of 6 values each)");
    std::vector<std::array<double, 6>> sv(nsrc);
    for (int m = 0; m < nsrc; ++m)
        for (int i = 0; i < 6; ++i) {
            sv[m][i] = src[m * 6 + i];
            if (!std::isfinite(sv[m][i])) return fail(FR_EINVAL, "non-finite source parameter");
        }
    for (const auto& v : sv)
        if (!(v[1] >= 0.0)) return fail(FR_EINVAL, "source range factor k must be >= 0");
    if (nsrc > 0 && !c->order.empty())
        for (int32_t q : c->order[cand])
            if (q < c->p) return fail(FR_EINVAL, "the energy source needs a candidate of uniform degree");
    CK(cudaDeviceSynchronize());
    if (!c->tnow) {
        const size_t nc = size_t(c->ncand);
        if (cudaMalloc(&c->tnow, nc * 8) != cudaSuccess ||
            cudaMalloc(&c->src_A, nc * frk::MAXSRC * 8) != cudaSuccess ||
            cudaMalloc(&c->src_f, nc * frk::MAXSRC * 8) != cudaSuccess)
            return fail(FR_ENOMEM, "cannot allocate source tables");
        CK(cudaMemset(c->tnow, 0, nc * 8));
    }
    if (!c->dtc) {
        const size_t nc = size_t(c->ncand);
        if (cudaMalloc(&c->dtc, nc * 8) != cudaSuccess) return fail(FR_ENOMEM, "cannot allocate source tables");
        CK(cudaMemcpy(c->dtc, c->cand_dt.data(), nc * 8, cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(c->tnow + cand, &t0, 8, cudaMemcpyHostToDevice));
    c->srcs[cand] = sv;
    const int rc = rebuild_sources(c);
    if (rc) return fail(rc, "cannot build the source table");
    invalidate_graph(c);
    CK(cudaDeviceSynchronize());
    return FR_OK;
}

extern "C" int fr_set_element_order(fr_ctx* c, int cand, const int32_t* order) {
    if (!c || cand < -1 || cand >= c->ncand) return fail(FR_EINVAL, "bad argument");
    const int k0 = cand < 0 ? 0 : cand, k1 = cand < 0 ? c->ncand : cand + 1;
    if (order) {
        const int64_t n = c->cand_off[k1] - c->cand_off[k0];
        for (int64_t i = 0; i < n; ++i)
            if (order[i] < 0 || order[i] > c->p) return fail(FR_EINVAL, "element order outside 0..p");
        for (int k = k0; k < k1; ++k) {
            if (c->srcs.empty() || c->srcs[k].empty()) continue;
            for (int64_t e = c->cand_off[k]; e < c->cand_off[k + 1]; ++e)
                if (order[e - c->cand_off[k0]] < c->p)
                    return fail(FR_EINVAL, "the energy source needs a candidate of uniform degree");
        }
    }
    CK(cudaDeviceSynchronize());
    if (c->order.empty()) c->order.resize(c->ncand);
    for (int k = k0; k < k1; ++k) {
        const int64_t a0 = c->cand_off[k], n = c->cand_off[k + 1] - a0;
        if (order) c->order[k].assign(order + (a0 - c->cand_off[k0]), order + (a0 - c->cand_off[k0]) + n);
        else c->order[k].clear();
    }
    // the device list: (element, cap) of every element with cap < p, by candidate
    std::vector<int32_t> el, cp;
    c->sp_off.assign(c->ncand + 1, 0);
    for (int k = 0; k < c->ncand; ++k) {
        for (size_t i = 0; i < c->order[k].size(); ++i)
            if (c->order[k][i] < c->p) {
                el.push_back(int32_t(c->cand_off[k] + int64_t(i)));
                cp.push_back(c->order[k][i]);
            }
        c->sp_off[k + 1] = int(el.size());
    }
    for (int32_t** b : {&c->sp_elem, &c->sp_cap}) {
        if (*b) cudaFree(*b);
        *b = nullptr;
    }
    c->sp_n = 0;
    if (!el.empty()) {
        const size_t bytes = el.size() * sizeof(int32_t);
        if (cudaMalloc(&c->sp_elem, bytes) != cudaSuccess || cudaMalloc(&c->sp_cap, bytes) != cudaSuccess)
            return fail(FR_ENOMEM, "cannot allocate the element order table");
        CK(cudaMemcpy(c->sp_elem, el.data(), bytes, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->sp_cap, cp.data(), bytes, cudaMemcpyHostToDevice));
        c->sp_n = int(el.size());
        // the current state of the changed candidates moves into the reduced spaces
        for (int k = k0; k < k1; ++k) {
            const int rc = c->prec == FR_FP64
                               ? L_sponge<double>(c, static_cast<double*>(c->u0), nullptr, nullptr, nullptr, k)
                               : L_sponge<float>(c, static_cast<float*>(c->u0), nullptr, nullptr, nullptr, k);
            CKL(rc, "sponge kernel");
        }
    }
    CK(cudaDeviceSynchronize());
    const int rc = build_reduced(c);
    if (rc) return fail(rc, "cannot build the reduced-degree element tables");
    c->traces_valid = false;
    invalidate_graph(c);
    CK(cudaDeviceSynchronize());
    return FR_OK;
}

// per-element and per-candidate step buffers (filled with the current steps)
int ensure_dt_buffers(fr_ctx* c) {
    const size_t nc = size_t(c->ncand);
    if (!c->dtc) {
        if (cudaMalloc(&c->dtc, nc * 8) != cudaSuccess) return fail(FR_ENOMEM, "cannot allocate step buffers");
        CK(cudaMemcpy(c->dtc, c->cand_dt.data(), nc * 8, cudaMemcpyHostToDevice));
    }
    if (!c->dte) {
        if (cudaMalloc(&c->dte, size_t(c->E) * c->rsz) != cudaSuccess) {
            c->dte = nullptr;
            return fail(FR_ENOMEM, "cannot allocate per-element time steps");
        }
        for (int k = 0; k < c->ncand; ++k) {
            const int64_t a0 = c->cand_off[k], n = c->cand_off[k + 1] - a0;
            if (c->prec == FR_FP64) k_fill_d<<<256, 256>>>(static_cast<double*>(c->dte) + a0, n, c->cand_dt[k]);
            else k_fill_f<<<256, 256>>>(static_cast<float*>(c->dte) + a0, n, float(c->cand_dt[k]));
            c->launches += 1;
        }
        CK(cudaGetLastError());
    }
    if (!c->lam && cudaMalloc(&c->lam, nc * sizeof(unsigned long long)) != cudaSuccess)
        return fail(FR_ENOMEM, "cannot allocate step buffers");
    return FR_OK;
}

extern "C" int fr_set_adaptive_dt(fr_ctx* c, double cfl) {
    if (!c || !std::isfinite(cfl)) return fail(FR_EINVAL, "bad argument");
    CK(cudaDeviceSynchronize());
    if (cfl > 0.0) {
        const int rc = ensure_dt_buffers(c);
        if (rc) return rc;
    } else if (c->adaptive_cfl > 0.0) {
        // back to the fixed steps of fr_set_cand_dt / the options
        for (int k = 0; k < c->ncand; ++k) {
            const int64_t a0 = c->cand_off[k], n = c->cand_off[k + 1] - a0;
            if (c->prec == FR_FP64) k_fill_d<<<256, 256>>>(static_cast<double*>(c->dte) + a0, n, c->cand_dt[k]);
            else k_fill_f<<<256, 256>>>(static_cast<float*>(c->dte) + a0, n, float(c->cand_dt[k]));
            c->launches += 1;
        }
        CK(cudaMemcpy(c->dtc, c->cand_dt.data(), size_t(c->ncand) * 8, cudaMemcpyHostToDevice));
    }
    c->adaptive_cfl = cfl > 0.0 ? cfl : 0.0;
    invalidate_graph(c);
    CK(cudaDeviceSynchronize());
    return FR_OK;
}

extern "C" int fr_cand_dt(const fr_ctx* c, int cand, double* dt) {
    if (!c || !dt || cand < 0 || cand >= c->ncand) return fail(FR_EINVAL, "bad argument");
    if (!c->dtc) {
        *dt = c->cand_dt[cand];
        return FR_OK;
    }
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(dt, c->dtc + cand, 8, cudaMemcpyDeviceToHost));
    return FR_OK;
}

extern "C" int fr_source_time(const fr_ctx* c, int cand, double* t) {
    if (!c || !t || cand < 0 || cand >= c->ncand) return fail(FR_EINVAL, "bad argument");
    *t = 0.0;
    if (!c->tnow) return FR_OK;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(t, c->tnow + cand, 8, cudaMemcpyDeviceToHost));
    return FR_OK;
}

extern "C" int fr_forces(fr_ctx* c, int cand, double out[5]) {
    if (!c || !out || cand < 0 || cand >= c->ncand) return fail(FR_EINVAL, "bad argument");
    CK(cudaDeviceSynchronize());
    double fnow[3], fsum[3], cnt;
    CK(cudaMemcpy(fnow, c->fnow + 3 * cand, sizeof(fnow), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(fsum, c->fsum + 3 * cand, sizeof(fsum), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&cnt, c->fcnt + cand, sizeof(double), cudaMemcpyDeviceToHost));
    const fr_options& o = c->opt;
    double v2 = 0;
    for (int i = 0; i < c->dim; ++i) v2 += o.vel_inf[i] * o.vel_inf[i];
    const double qa = 0.5 * o.rho_inf * v2 * o.ref_area;
    if (!(qa > 0.0)) return fail(FR_EINVAL, "force coefficients need |V_inf| > 0 and ref_area > 0");
    double cl = 0, cd = 0, ml = 0, md = 0;
    for (int i = 0; i < c->dim; ++i) {
        cl += fnow[i] * o.lift_dir[i];
        cd += fnow[i] * o.drag_dir[i];
        ml += fsum[i] * o.lift_dir[i];
        md += fsum[i] * o.drag_dir[i];
    }
    out[0] = cl / qa;
    out[1] = cd / qa;
    out[2] = cnt > 0 ? ml / (qa * cnt) : 0.0;
    out[3] = cnt > 0 ? md / (qa * cnt) : 0.0;
    out[4] = cnt;
    int bad = 0;
    CK(cudaMemcpy(&bad, c->nonfinite + cand, sizeof(int), cudaMemcpyDeviceToHost));
    if (bad) return fail(FR_ENONFINITE, "candidate " + std::to_string(cand) + ": a step produced NaN or Inf");
    return FR_OK;
}

extern "C" int fr_forces_reset(fr_ctx* c) {
    if (!c) return fail(FR_EINVAL, "null argument");
    CK(cudaDeviceSynchronize());
    CK(cudaMemset(c->fsum, 0, sizeof(double) * 3 * c->ncand));
    CK(cudaMemset(c->fcnt, 0, sizeof(double) * c->ncand));
    return FR_OK;
}

extern "C" int fr_integrals(fr_ctx* c, int cand, double* out) {
    if (!c || !out) return fail(FR_EINVAL, "null argument");
    int64_t first, count;
    int rc = fr_cand_range(c, cand, &first, &count);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    const int nb = int(std::min<int64_t>(c->partial_blocks, std::max<int64_t>(1, (count * c->nsp + 255) / 256)));
    if (c->prec == FR_FP64) {
        auto g = geo_of<double>(c);
        const auto& op = c->opd;
        rc = c->dim == 2 ? frl::integrals<double, 2>(c->p, static_cast<const double*>(c->u0), first, count, op, g,
                                                     c->partial, nb, nullptr)
                         : frl::integrals<double, 3>(c->p, static_cast<const double*>(c->u0), first, count, op, g,
                                                     c->partial, nb, nullptr);
    } else {
        auto g = geo_of<float>(c);
        const auto& op = c->opf;
        rc = c->dim == 2 ? frl::integrals<float, 2>(c->p, static_cast<const float*>(c->u0), first, count, op, g,
                                                    c->partial, nb, nullptr)
                         : frl::integrals<float, 3>(c->p, static_cast<const float*>(c->u0), first, count, op, g,
                                                    c->partial, nb, nullptr);
    }
    ++c->launches;
    CKL(rc, "integrals kernel");
    std::vector<double> h(size_t(nb) * (c->nv + 1));
    CK(cudaMemcpy(h.data(), c->partial, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int v = 0; v <= c->nv; ++v) {
        double s = 0;
        for (int b = 0; b < nb; ++b) s += h[size_t(b) * (c->nv + 1) + v];
        out[v] = s;
    }
    return FR_OK;
}

// ---------------------------------------------------------------- FW-H surfaces
extern "C" int fwh_register(fr_ctx* c, int cand, int npts, const double* xyz, int capacity, int every,
                            int* handle) {
    if (!c || !xyz || !handle || npts < 1 || capacity < 1 || every < 1 || cand < 0 || cand >= c->ncand)
        return fail(FR_EINVAL, "bad argument");
    const int dim = c->dim;
    const int q = c->q[cand];
    const int nq = q + 1;
    const int nn = dim == 2 ? nq * nq : nq * nq * nq;
    const int64_t ne = c->cand_off[cand + 1] - c->cand_off[cand];
    const double* nodes = c->nodes[cand].data();
    // element bounding boxes, binned on a uniform grid
    std::vector<double> lo(ne * dim), hi(ne * dim);
    double glo[3] = {1e300, 1e300, 1e300}, ghi[3] = {-1e300, -1e300, -1e300};
    for (int64_t e = 0; e < ne; ++e)
        for (int i = 0; i < dim; ++i) {
            double a = 1e300, b = -1e300;
            for (int k = 0; k < nn; ++k) {
                a = std::min(a, nodes[(e * nn + k) * dim + i]);
                b = std::max(b, nodes[(e * nn + k) * dim + i]);
            }
            const double pad = 0.05 * (b - a) + 1e-12;
            lo[e * dim + i] = a - pad;
            hi[e * dim + i] = b + pad;
            glo[i] = std::min(glo[i], a - pad);
            ghi[i] = std::max(ghi[i], b + pad);
        }
    const int G = std::max(1, int(std::pow(double(ne), 1.0 / dim)));
    auto cell = [&](int i, double x) {
        int k = int((x - glo[i]) / (ghi[i] - glo[i]) * G);
        return std::min(G - 1, std::max(0, k));
    };
    const int ncell = dim == 2 ? G * G : G * G * G;
    std::vector<std::vector<int64_t>> bins(ncell);
    for (int64_t e = 0; e < ne; ++e) {
        int a[3], b[3];
        for (int i = 0; i < 3; ++i) { a[i] = 0; b[i] = 0; }
        for (int i = 0; i < dim; ++i) {
            a[i] = cell(i, lo[e * dim + i]);
            b[i] = cell(i, hi[e * dim + i]);
        }
        for (int z = a[2]; z <= b[2]; ++z)
            for (int y = a[1]; y <= b[1]; ++y)
                for (int x = a[0]; x <= b[0]; ++x) bins[(z * G + y) * G + x].push_back(e);
    }
    std::vector<int64_t> pe(npts);
    std::vector<double> pw(size_t(npts) * dim * c->np);
    for (int k = 0; k < npts; ++k) {
        const double* y = xyz + size_t(k) * 3;
        int ci[3] = {0, 0, 0};
        for (int i = 0; i < dim; ++i) ci[i] = cell(i, y[i]);
        const auto& list = bins[(ci[2] * G + ci[1]) * G + ci[0]];
        int64_t found = -1;
        double xi[3] = {0, 0, 0};
        for (int64_t e : list) {
            bool inside = true;
            for (int i = 0; i < dim; ++i)
                if (y[i] < lo[e * dim + i] || y[i] > hi[e * dim + i]) inside = false;
            if (!inside) continue;
            double t[3] = {0, 0, 0};
            bool ok = false;
            for (int it = 0; it < 50; ++it) {
                double x[3], A[9];
                frg::element_map(dim, q, nodes + e * nn * dim, t, x, A);
                double r[3] = {y[0] - x[0], y[1] - x[1], dim == 3 ? y[2] - x[2] : 0.0};
                double d[3];
                if (dim == 2) {
                    const double det = A[0] * A[3] - A[1] * A[2];
                    d[0] = (A[3] * r[0] - A[1] * r[1]) / det;
                    d[1] = (-A[2] * r[0] + A[0] * r[1]) / det;
                } else {
                    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                                       A[2] * (A[3] * A[7] - A[4] * A[6]);
                    d[0] = (r[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (r[1] * A[8] - A[5] * r[2]) +
                            A[2] * (r[1] * A[7] - A[4] * r[2])) / det;
                    d[1] = (A[0] * (r[1] * A[8] - A[5] * r[2]) - r[0] * (A[3] * A[8] - A[5] * A[6]) +
                            A[2] * (A[3] * r[2] - r[1] * A[6])) / det;
                    d[2] = (A[0] * (A[4] * r[2] - r[1] * A[7]) - A[1] * (A[3] * r[2] - r[1] * A[6]) +
                            r[0] * (A[3] * A[7] - A[4] * A[6])) / det;
                }
                double dm = 0, tm = 0;
                for (int i = 0; i < dim; ++i) {
                    t[i] += d[i];
                    dm = std::max(dm, std::fabs(d[i]));
                    tm = std::max(tm, std::fabs(t[i]));
                }
                if (!(tm < 3.0)) break;
                if (dm < 1e-13) {
                    ok = true;
                    break;
                }
            }
            bool in = ok;
            for (int i = 0; i < dim; ++i) in = in && std::fabs(t[i]) <= 1.0 + 1e-10;
            if (in) {
                found = e;
                for (int i = 0; i < dim; ++i) xi[i] = std::max(-1.0, std::min(1.0, t[i]));
                break;
            }
        }
        if (found < 0) return fail(FR_EINVAL, "surface point " + std::to_string(k) + " is outside the mesh");
        pe[k] = c->cand_off[cand] + found;
        for (int i = 0; i < dim; ++i)
            for (int j = 0; j < c->np; ++j)
                pw[(size_t(k) * dim + i) * c->np + j] = frg::lagrange(c->ref.x, c->np, j, xi[i]);
    }
    Surface sf;
    sf.cand = cand;
    sf.npts = npts;
    sf.cap = capacity;
    sf.every = every;
    int rc;
    if ((rc = upload(reinterpret_cast<void**>(&sf.pe), pe)) || (rc = upload_real(&sf.pw, pw, c->prec))) return rc;
    if (cudaMalloc(&sf.hist, size_t(capacity) * npts * 5 * c->rsz) != cudaSuccess ||
        cudaMalloc(&sf.count, 3 * sizeof(int)) != cudaSuccess) {
        if (sf.hist) cudaFree(sf.hist);
        cudaFree(sf.pe);
        cudaFree(sf.pw);
        return fail(FR_ENOMEM, "cannot allocate the FW-H history");
    }
    CK(cudaMemset(sf.count, 0, 3 * sizeof(int)));
    c->surf.push_back(sf);
    invalidate_graph(c);
    *handle = int(c->surf.size()) - 1;
    return FR_OK;
}

extern "C" int fwh_sample(fr_ctx* c, int handle, void* stream) {
    if (!c || handle < 0 || handle >= int(c->surf.size())) return fail(FR_EINVAL, "bad surface handle");
    Surface& sf = c->surf[handle];
    int cnt[3] = {0, 0, 0};
    CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    CK(cudaMemcpy(cnt, sf.count, sizeof(cnt), cudaMemcpyDeviceToHost));
    if (cnt[0] >= sf.cap) return fail(FR_EINVAL, "FW-H history is full");
    // an explicit sample is taken now: align the step phase, then restore it
    const int phase = cnt[1];
    int aligned[3] = {cnt[0], 0, cnt[2]};
    CK(cudaMemcpy(sf.count, aligned, sizeof(aligned), cudaMemcpyHostToDevice));
    const int rc = c->prec == FR_FP64 ? L_sample<double>(c, sf, static_cast<cudaStream_t>(stream))
                                      : L_sample<float>(c, sf, static_cast<cudaStream_t>(stream));
    CKL(rc, "sampling kernel");
    CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    CK(cudaMemcpy(&aligned, sf.count, sizeof(aligned), cudaMemcpyDeviceToHost));
    aligned[1] = phase;
    CK(cudaMemcpy(sf.count, aligned, sizeof(aligned), cudaMemcpyHostToDevice));
    return FR_OK;
}

extern "C" int fwh_history(fr_ctx* c, int handle, double* out, int* nrec) {
    if (!c || !nrec || handle < 0 || handle >= int(c->surf.size())) return fail(FR_EINVAL, "bad argument");
    Surface& sf = c->surf[handle];
    CK(cudaDeviceSynchronize());
    int ctr[3] = {0, 0, 0};
    CK(cudaMemcpy(ctr, sf.count, sizeof(ctr), cudaMemcpyDeviceToHost));
    const int cnt = ctr[0], over = ctr[2];
    *nrec = cnt;
    if (!out) return over ? fail(FR_EINVAL, "FW-H history overflowed") : FR_OK;
    const size_t n = size_t(cnt) * sf.npts * 5;
    std::vector<double> h(n);
    if (c->prec == FR_FP64) {
        CK(cudaMemcpy(h.data(), sf.hist, n * 8, cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> f(n);
        CK(cudaMemcpy(f.data(), sf.hist, n * 4, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) h[i] = f[i];
    }
    const fr_options& o = c->opt;
    for (size_t r = 0; r < size_t(cnt) * sf.npts; ++r) {
        out[r * 5 + 0] = h[r * 5 + 0] + o.rho_inf;
        for (int i = 0; i < 3; ++i) out[r * 5 + 1 + i] = h[r * 5 + 1 + i] + (i < c->dim ? o.vel_inf[i] : 0.0);
        out[r * 5 + 4] = h[r * 5 + 4] + o.p_inf;
    }
    return over ? fail(FR_EINVAL, "FW-H history overflowed") : FR_OK;
}

extern "C" int fwh_clear(fr_ctx* c, int handle) {
    if (!c || handle < 0 || handle >= int(c->surf.size())) return fail(FR_EINVAL, "bad surface handle");
    CK(cudaDeviceSynchronize());
    CK(cudaMemset(c->surf[handle].count, 0, 3 * sizeof(int)));
    return FR_OK;
}

// ---------------------------------------------------------------- tiles
extern "C" int fr_set_tile(fr_ctx* c, int epb) {
    if (!c || epb < 0 || epb > 32) return fail(FR_EINVAL, "bad tile (elements per block 0..32)");
    if (epb > max_epb(c))
        return fail(FR_EINVAL, "bad tile: at most " + std::to_string(max_epb(c)) + " elements per block at this order");
    if (epb == 0) {
        default_launch(c);
    } else {
        for (int k = 0; k < 3; ++k)
            if (smem_of(c, k, epb) > 227 * 1024) return fail(FR_EINVAL, "tile needs too much shared memory");
        for (int k = 0; k < 3; ++k) {
            c->lc[k].epb = epb;
            c->lc[k].threads = tpe_of(c) * epb;
        }
    }
    invalidate_graph(c);
    return FR_OK;
}

extern "C" int fr_autotune(fr_ctx* c, int* best) {
    if (!c) return fail(FR_EINVAL, "null argument");
    // time each sweep for 1..16 elements (warps) per block on the current
    // state; keep the fastest per kernel.  Results do not depend on the tile.
    const int cand[] = {1, 2, 4, 8, 16};
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    frk::Launch bestl[3] = {c->lc[0], c->lc[1], c->lc[2]};
    float bestt[3] = {1e30f, 1e30f, 1e30f};
    // scratch for a stage-2-like residual launch (reads u0 and acc, writes acc,
    // the stage output and the next traces), as the step runs it
    void *R = nullptr, *A = nullptr, *TR = nullptr;
    const size_t nstate = size_t(c->E) * c->nv * c->nsp * c->rsz;
    const size_t ntrace = size_t(c->E) * c->nf * c->nv * c->nfp * c->rsz;
    if (cudaMalloc(&R, nstate) != cudaSuccess || cudaMalloc(&A, nstate) != cudaSuccess ||
        cudaMalloc(&TR, ntrace) != cudaSuccess) {
        if (R) cudaFree(R);
        if (A) cudaFree(A);
        return fail(FR_ENOMEM, "autotune scratch");
    }
    CK(cudaMemset(A, 0, nstate));
    c->traces_valid = false;
    for (int epb : cand) {
        bool fits = true;
        for (int k = 0; k < 3; ++k) fits = fits && smem_of(c, k, epb) <= 200 * 1024;
        fits = fits && epb <= max_epb(c);
        if (!fits) continue;
        for (int k = 0; k < 3; ++k) c->lc[k] = frk::Launch{epb, tpe_of(c) * epb};
        for (int kern = 0; kern < 3; ++kern) {
            if (kern == 1 && !c->visc) continue;
            float tot = 1e30f;   // best of the timed repetitions
            int rc = 0;
            for (int rep = 0; rep < 12 && rc == 0; ++rep) {
                CK(cudaEventRecord(a, nullptr));
                if (c->prec == FR_FP64) {
                    const double* u = static_cast<const double*>(c->u0);
                    double* uf = static_cast<double*>(c->ufb[0]);
                    if (kern == 0) rc = L_traces<double>(c, u, uf, nullptr);
                    else if (kern == 1) rc = L_visc<double>(c, u, uf, nullptr);
                    else {
                        frk::Stage<double> st{2, 0.0, nullptr, nullptr, static_cast<double*>(c->u0),
                                              static_cast<double*>(R), static_cast<double*>(A),
                                              static_cast<double*>(TR)};
                        rc = L_resid<double>(c, u, uf, st, nullptr);
                    }
                } else {
                    const float* u = static_cast<const float*>(c->u0);
                    float* uf = static_cast<float*>(c->ufb[0]);
                    if (kern == 0) rc = L_traces<float>(c, u, uf, nullptr);
                    else if (kern == 1) rc = L_visc<float>(c, u, uf, nullptr);
                    else {
                        frk::Stage<float> st{2, 0.0f, nullptr, nullptr, static_cast<float*>(c->u0),
                                             static_cast<float*>(R), static_cast<float*>(A),
                                             static_cast<float*>(TR)};
                        rc = L_resid<float>(c, u, uf, st, nullptr);
                    }
                }
                CK(cudaEventRecord(b, nullptr));
                CK(cudaEventSynchronize(b));
                float ms = 0;
                cudaEventElapsedTime(&ms, a, b);
                if (rep > 0) tot = std::min(tot, ms);
            }
            if (rc == 0 && tot > 0 && tot < 1e30f && tot < bestt[kern]) {
                bestt[kern] = tot;
                bestl[kern] = frk::Launch{epb, tpe_of(c) * epb};
            }
        }
    }
    for (int k = 0; k < 3; ++k) c->lc[k] = bestl[k];
    cudaFree(R);
    cudaFree(A);
    cudaFree(TR);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    c->traces_valid = false;
    invalidate_graph(c);
    if (best) *best = c->lc[2].epb;
    return FR_OK;
}

extern "C" int64_t fr_launch_count(const fr_ctx* c) { return c ? c->launches : 0; }

// Independent FMA chains per thread; the result is stored so nothing is elided.
__global__ void k_dfma_probe(double* out, int iters, double a, double b) {
    double x0 = threadIdx.x * 1e-9, x1 = x0 + 1e-3, x2 = x0 + 2e-3, x3 = x0 + 3e-3;
    double x4 = x0 + 4e-3, x5 = x0 + 5e-3, x6 = x0 + 6e-3, x7 = x0 + 7e-3;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

extern "C" int fr_probe_fp64_peak(double* gflops, void* stream) {
    if (!gflops) return fail(FR_EINVAL, "null argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256, iters = 4096;
    double* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return fail(FR_ENOMEM, "probe buffer");
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_dfma_probe<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-7);  // warm-up
    cudaEventRecord(a, s);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) k_dfma_probe<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(b, s);
    const cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    if (e != cudaSuccess) return fail(FR_ECUDA, cudaGetErrorString(e));
    const double flops = 2.0 * 8.0 * double(iters) * blocks * threads * reps;
    *gflops = flops / (double(ms) * 1e-3) / 1e9;
    return FR_OK;
}

extern "C" int fr_profile_step(fr_ctx* c, int nsteps, void* stream, double ms_out[6], int64_t n_out[6]) {
    if (!c || nsteps < 0 || !ms_out || !n_out) return fail(FR_EINVAL, "bad argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int k = 0; k < 6; ++k) {
        ms_out[k] = 0.0;
        n_out[k] = 0;
    }
    // traces of a state set from outside (outside the graph, as in fr_rk_step_graph)
    {
        Prof p0;
        p0.s = s;
        const int rc = c->prec == FR_FP64 ? ensure_traces<double>(c, s, &p0) : ensure_traces<float>(c, s, &p0);
        CK(cudaStreamSynchronize(s));
        for (size_t i = 0; i < p0.kind.size() && 2 * i + 1 < p0.ev.size(); ++i) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, p0.ev[2 * i], p0.ev[2 * i + 1]);
            ms_out[p0.kind[i]] += ms;
            n_out[p0.kind[i]] += 1;
        }
        for (auto ev : p0.ev) cudaEventDestroy(ev);
        if (rc) return rc;
    }
    // one step captured with event record nodes around every kernel, replayed
    // nsteps times: the same launch sequence as fr_rk_step_graph
    Prof pr;
    pr.s = c->cap_stream;
    pr.external = true;
    const int64_t before = c->launches;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = c->prec == FR_FP64 ? enqueue_step<double>(c, c->cap_stream, &pr)
                                      : enqueue_step<float>(c, c->cap_stream, &pr);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c->cap_stream, &graph);
    const int64_t per_step = c->launches - before;
    c->launches = before;
    cudaGraphExec_t gx = nullptr;
    cudaError_t e = ec;
    if (rc == FR_OK && ec == cudaSuccess) e = cudaGraphInstantiate(&gx, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    for (int k = 0; k < nsteps && rc == FR_OK && e == cudaSuccess; ++k) {
        e = cudaGraphLaunch(gx, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        c->launches += per_step;
        for (size_t i = 0; i < pr.kind.size() && 2 * i + 1 < pr.ev.size(); ++i) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, pr.ev[2 * i], pr.ev[2 * i + 1]);
            ms_out[pr.kind[i]] += ms;
            n_out[pr.kind[i]] += 1;
        }
    }
    if (gx) cudaGraphExecDestroy(gx);
    for (auto ev : pr.ev) cudaEventDestroy(ev);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(FR_ECUDA, std::string("profile graph: ") + cudaGetErrorString(e));
    return FR_OK;
}
