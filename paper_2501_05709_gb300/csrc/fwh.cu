// FW-H acoustic pressure at far-field observers from a stationary permeable
// data surface in a uniformly moving medium (Appendix B, Eqs. B.2-B.14),
// advanced-time (source-time-dominant) form, in double precision.
//
//   k_fwh_series : per panel and source time, the thickness and loading
//                  sources Q (Eq. A.5) and L_i (Eqs. A.7-A.8, sigma_ij
//                  omitted), with u_i the disturbance velocity V - U_inf,
//                  and their 4th-order finite-difference tau-derivatives.
//   k_fwh_accum  : per (panel, spanwise copy) the radii R*, R and their
//                  gradients (Eqs. B.8-B.12) give the integrand coefficients
//                  of Eqs. B.2-B.3; each observer time t* (unified window,
//                  step dtau) interpolates the panel integrand at
//                  tau = t* - R/c0 (Eq. B.13) with a 4-point cubic Lagrange
//                  stencil and sums (Eq. B.14); one partial row per panel group.
//   k_fwh_reduce : sums the partial rows in a fixed order, divides by 4 pi.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "fr.h"

namespace {

constexpr int NSER = 8;  // Q, L1, L2, L3, dQ, dL1, dL2, dL3

struct FwhConst {
    double M[3];
    double c0, rho0, p0, dtau, tau0;
    double b2;  // Prandtl-Glauert factor squared, 1 / (1 - |M|^2)
};

__device__ __forceinline__ void sources(const double* h, const double* n, const FwhConst& k, double* out) {
    // h = (rho, V1, V2, V3, p) total; disturbance u = V - c0 M
    double u[3];
    double un = 0.0, Un = 0.0;
    for (int i = 0; i < 3; ++i) {
        u[i] = h[1 + i] - k.c0 * k.M[i];
        un += u[i] * n[i];
        Un += k.c0 * k.M[i] * n[i];
    }
    const double rho = h[0];
    out[0] = rho * (un + Un) - k.rho0 * Un;
    for (int i = 0; i < 3; ++i) out[1 + i] = (h[4] - k.p0) * n[i] + rho * u[i] * (un + Un);
}

__global__ void k_fwh_series(const double* __restrict__ hist, int nt, int npts, const double* __restrict__ nrm,
                             FwhConst k, double* __restrict__ X) {
    const int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (w >= int64_t(nt) * npts) return;
    const int p = int(w % npts);
    const int t = int(w / npts);
    const double n[3] = {nrm[p * 3 + 0], nrm[p * 3 + 1], nrm[p * 3 + 2]};
    // the 5-point stencil: central inside, one-sided 4th order at both ends
    int j0;
    double c[5];
    const double s = 1.0 / (12.0 * k.dtau);
    if (t >= 2 && t <= nt - 3) {
        j0 = t - 2;
        c[0] = 1; c[1] = -8; c[2] = 0; c[3] = 8; c[4] = -1;
    } else if (t == 0) {
        j0 = 0;
        c[0] = -25; c[1] = 48; c[2] = -36; c[3] = 16; c[4] = -3;
    } else if (t == 1) {
        j0 = 0;
        c[0] = -3; c[1] = -10; c[2] = 18; c[3] = -6; c[4] = 1;
    } else if (t == nt - 1) {
        j0 = nt - 5;
        c[0] = 3; c[1] = -16; c[2] = 36; c[3] = -48; c[4] = 25;
    } else {
        j0 = nt - 5;
        c[0] = -1; c[1] = 6; c[2] = -18; c[3] = 10; c[4] = 3;
    }
    double here[4], der[4] = {0, 0, 0, 0};
    sources(hist + (int64_t(t) * npts + p) * 5, n, k, here);
    for (int m = 0; m < 5; ++m) {
        double q[4];
        sources(hist + (int64_t(j0 + m) * npts + p) * 5, n, k, q);
        for (int v = 0; v < 4; ++v) der[v] += c[m] * q[v];
    }
    double* xp = X + int64_t(p) * NSER * nt;
    for (int v = 0; v < 4; ++v) {
        xp[v * nt + t] = here[v];
        xp[(4 + v) * nt + t] = der[v] * s;
    }
}

// Geometry of one (panel, copy): integrand coefficients and delay.
__device__ void panel_coefs(const double* y, double dS, const double* obs, const FwhConst& k, double* cf,
                            double* delay) {
    double r[3];
    for (int i = 0; i < 3; ++i) r[i] = obs[i] - y[i];
    double Mr = 0, rr = 0, MM = 0;
    for (int i = 0; i < 3; ++i) {
        Mr += k.M[i] * r[i];
        rr += r[i] * r[i];
        MM += k.M[i] * k.M[i];
    }
    (void)MM;
    const double b2 = k.b2;
    const double Rs = sqrt(rr + b2 * Mr * Mr) / sqrt(b2);          // Eq. B.8
    const double R = b2 * (Rs - Mr);                               // Eq. B.9
    double Rts[3], Rt[3];
    double MRs = 0, MR = 0;
    for (int i = 0; i < 3; ++i) {
        Rts[i] = (r[i] + b2 * Mr * k.M[i]) / (b2 * Rs);            // Eq. B.11
        Rt[i] = b2 * (Rts[i] - k.M[i]);                            // Eq. B.12
        MRs += k.M[i] * Rts[i];
        MR += k.M[i] * Rt[i];
    }
    // I = a dQ + b Q + sum_i (d_i dL_i + e_i L_i)   (Eqs. B.2-B.7, times dS)
    cf[4] = (1.0 - MR) * dS / Rs;
    cf[0] = -k.c0 * MRs * dS / (Rs * Rs);
    for (int i = 0; i < 3; ++i) {
        cf[5 + i] = Rt[i] * dS / (k.c0 * Rs);
        cf[1 + i] = Rts[i] * dS / (Rs * Rs);
    }
    *delay = R / k.c0;
}

// Each thread accumulates FWH_KO consecutive observer-time samples over the
// panel-copies of its block's group.  A panel-copy's stencil offset and cubic
// weights are the same for every sample (t = tstart + i dtau advances the
// source index by exactly 1 per sample), so they are computed once per block;
// each source time j in the thread's window combines the 8 series once
// (I_j = sum_v cf_v X_v(j)) and serves up to four samples.  Samples whose
// stencil is clamped at the ends of the record take the general per-sample
// path.  Small groups give many blocks per observer (the FP64 pipe needs the
// parallelism).
constexpr int FWH_KO = 4;
constexpr int kFwhGroup = 32;      // panel-copies per block (groups of whole panels)
constexpr int FWH_SH = NSER + 5;   // per panel-copy: cf[8], weights[4], source index of sample 0
// dynamic shared memory per panel-copy: the doubles above, the offset of the
// panel's series and the stencil start of sample 0 (integers, so that the
// sample loop does no FP64 conversions)
constexpr size_t FWH_SH_BYTES = sizeof(double) * FWH_SH + sizeof(int64_t) + sizeof(int);

__global__ void k_fwh_accum(const double* __restrict__ X, int nt, int npts, const double* __restrict__ y,
                            const double* __restrict__ dS, FwhConst k, double ox, double oy, double oz,
                            double tstart, int T, int ncopies, double Lspan, int group,
                            double* __restrict__ partial) {
    extern __shared__ double sh[];  // [cap][FWH_SH] doubles, then int64 [cap], then int [cap]
    const int p0 = blockIdx.x * group;     // grid x: panel groups, grid y: sample blocks
    const int np = min(group, npts - p0);
    const int npc = np * ncopies;
    const int cap = group * ncopies;
    int64_t* xoff = reinterpret_cast<int64_t*>(sh + size_t(cap) * FWH_SH);
    int* jbs = reinterpret_cast<int*>(xoff + cap);
    const int K = (ncopies - 1) / 2;
    const double obs[3] = {ox, oy, oz};
    for (int w = threadIdx.x; w < npc; w += blockDim.x) {
        const int p = p0 + w / ncopies;
        const int cc = w % ncopies - K;
        const double yy[3] = {y[p * 3 + 0], y[p * 3 + 1], y[p * 3 + 2] + cc * Lspan};
        double delay;
        double* cf = sh + w * FWH_SH;
        panel_coefs(yy, dS[p], obs, k, cf, &delay);
        const double off = (tstart - k.tau0 - delay) / k.dtau;   // source index of sample 0
        const double fl = floor(off);
        const double x = off - fl + 1.0;                        // position in the stencil, [1, 2)
        cf[NSER + 0] = -(x - 1.0) * (x - 2.0) * (x - 3.0) / 6.0;
        cf[NSER + 1] = x * (x - 2.0) * (x - 3.0) / 2.0;
        cf[NSER + 2] = -x * (x - 1.0) * (x - 3.0) / 2.0;
        cf[NSER + 3] = x * (x - 1.0) * (x - 2.0) / 6.0;
        cf[NSER + 4] = off;
        jbs[w] = int(fl) - 1;
        xoff[w] = int64_t(p) * NSER * nt;
    }
    __syncthreads();
    const int i0 = (blockIdx.y * blockDim.x + threadIdx.x) * FWH_KO;
    if (i0 >= T) return;
    double acc[FWH_KO];
#pragma unroll
    for (int q = 0; q < FWH_KO; ++q) acc[q] = 0.0;
    const bool whole = i0 + FWH_KO <= T;
    for (int w = 0; w < npc; ++w) {
        const double* cf = sh + w * FWH_SH;
        const int j0 = i0 + jbs[w];
        const double* xp = X + xoff[w];
        if (whole && j0 >= 0 && j0 + FWH_KO + 3 <= nt) {
            double c[FWH_KO + 3];
#pragma unroll
            for (int m = 0; m < FWH_KO + 3; ++m) {
                double Ik = 0.0;
#pragma unroll
                for (int v = 0; v < NSER; ++v) Ik += cf[v] * xp[v * nt + j0 + m];
                c[m] = Ik;
            }
#pragma unroll
            for (int q = 0; q < FWH_KO; ++q) {
                double sum = 0.0;
#pragma unroll
                for (int m = 0; m < 4; ++m) sum += cf[NSER + m] * c[q + m];
                acc[q] += sum;
            }
        } else {
            const double off = cf[NSER + 4];
            for (int q = 0; q < FWH_KO && i0 + q < T; ++q) {
                const double s = double(i0 + q) + off;
                int j = int(floor(s)) - 1;
                j = max(0, min(nt - 4, j));
                const double x = s - double(j);
                const double wt[4] = {-(x - 1.0) * (x - 2.0) * (x - 3.0) / 6.0, x * (x - 2.0) * (x - 3.0) / 2.0,
                                      -x * (x - 1.0) * (x - 3.0) / 2.0, x * (x - 1.0) * (x - 2.0) / 6.0};
                double sum = 0.0;
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    double Ik = 0.0;
#pragma unroll
                    for (int v = 0; v < NSER; ++v) Ik += cf[v] * xp[v * nt + j + m];
                    sum += wt[m] * Ik;
                }
                acc[q] += sum;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < FWH_KO; ++q)
        if (i0 + q < T) partial[int64_t(blockIdx.x) * T + i0 + q] = acc[q];
}

// p'(t_i) = (1/4 pi) sum over panel groups of the partial sums: 32 samples x
// 32 group slices per block, each slice summing groups g = slice (mod 32) in
// order, then a fixed-order tree over the slices (the same order every call)
__global__ void k_fwh_reduce(const double* __restrict__ partial, int ngroups, int T, double* __restrict__ out) {
    __shared__ double red[32][33];
    const int i = blockIdx.x * 32 + threadIdx.x;
    double s = 0.0;
    if (i < T)
        for (int g = threadIdx.y; g < ngroups; g += 32) s += partial[int64_t(g) * T + i];
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    for (int st = 16; st > 0; st >>= 1) {
        if (threadIdx.y < st) red[threadIdx.y][threadIdx.x] += red[threadIdx.y + st][threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.y == 0 && i < T) out[i] = red[0][threadIdx.x] / (4.0 * M_PI);
}

}  // namespace

// records the message returned by fr_last_error (defined with the context code)
int fr_set_error_from_fwh(int code, const char* msg);

namespace {

// Host-side plan of one FW-H integration: the constants of Eqs. B.8-B.12,
// every observer's unified window (Eq. B.13 and the text after it: from the
// latest first arrival to the earliest last arrival over all panel copies),
// and the panel grouping of the accumulation kernel.
struct FwhPlan {
    FwhConst k;
    std::vector<double> tstart;   // first unified time per observer
    std::vector<int> Tn;          // unified samples per observer
    int group = 1, ngroups = 1, Tmax = 0;
};

int fwh_plan(int nt, int npts, const double* y, const double* n, const double* dS, const double* hist, double dtau,
             double tau0, const double* obs, int nobs, const double Minf[3], double c0, double rho0, double p0,
             double Lspan, int ncopies, const double* p_out, int cap, const int* nt_out, const double* t0_out,
             cudaStream_t s, FwhPlan& pl) {
    if (!hist || !y || !n || !dS || !obs || !Minf || !p_out || !nt_out || !t0_out)
        return fr_set_error_from_fwh(FR_EINVAL, "null argument");
    if (nt < 5 || npts < 1 || nobs < 1 || cap < 1 || ncopies < 1 || ncopies % 2 == 0 || !(dtau > 0.0) ||
        !(c0 > 0.0))
        return fr_set_error_from_fwh(FR_EINVAL, "bad sizes (nt >= 5, odd ncopies, dtau > 0, c0 > 0 required)");
    const double MM = Minf[0] * Minf[0] + Minf[1] * Minf[1] + Minf[2] * Minf[2];
    if (!(MM < 1.0)) return fr_set_error_from_fwh(FR_EINVAL, "|Minf| must be below 1");
    FwhConst& k = pl.k;
    for (int i = 0; i < 3; ++i) k.M[i] = Minf[i];
    k.c0 = c0;
    k.rho0 = rho0;
    k.p0 = p0;
    k.dtau = dtau;
    k.tau0 = tau0;
    k.b2 = 1.0 / (1.0 - MM);
    // unified observer windows (host, double): needs panel positions
    std::vector<double> yh(size_t(npts) * 3);
    if (cudaMemcpyAsync(yh.data(), y, yh.size() * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fr_set_error_from_fwh(FR_ECUDA, "cannot read panel positions");
    const int K = (ncopies - 1) / 2;
    pl.tstart.assign(nobs, 0.0);
    pl.Tn.assign(nobs, 0);
    for (int o = 0; o < nobs; ++o) {
        double dmax = -1e300, dmin = 1e300;
        for (int p = 0; p < npts; ++p)
            for (int cc = -K; cc <= K; ++cc) {
                double r[3] = {obs[o * 3 + 0] - yh[p * 3 + 0], obs[o * 3 + 1] - yh[p * 3 + 1],
                               obs[o * 3 + 2] - (yh[p * 3 + 2] + cc * Lspan)};
                double Mr = 0, rr = 0;
                for (int i = 0; i < 3; ++i) {
                    Mr += Minf[i] * r[i];
                    rr += r[i] * r[i];
                }
                const double Rs = std::sqrt(rr + k.b2 * Mr * Mr) / std::sqrt(k.b2);
                const double d = k.b2 * (Rs - Mr) / c0;
                dmax = std::max(dmax, d);
                dmin = std::min(dmin, d);
            }
        const double ts = tau0 + dmax;
        const double te = tau0 + (nt - 1) * dtau + dmin;
        if (te < ts) return fr_set_error_from_fwh(FR_EWINDOW, "empty observer window");
        const int T = int(std::floor((te - ts) / dtau + 1e-9)) + 1;
        if (T > cap) return fr_set_error_from_fwh(FR_EWINDOW, "observer window longer than the output capacity");
        pl.tstart[o] = ts;
        pl.Tn[o] = T;
    }
    pl.group = std::max(1, kFwhGroup / ncopies);
    pl.ngroups = (npts + pl.group - 1) / pl.group;
    if ((cap + 128 * FWH_KO - 1) / (128 * FWH_KO) > 65535)
        return fr_set_error_from_fwh(FR_EINVAL, "observer window too long for one launch");
    pl.Tmax = *std::max_element(pl.Tn.begin(), pl.Tn.end());
    return FR_OK;
}

// Scratch of a plan: the source series X [npts][NSER][nt] and one partial-sum
// row per panel group [ngroups][Tmax], in doubles.
size_t fwh_series_doubles(int npts, int nt) { return size_t(npts) * NSER * nt; }
size_t fwh_partial_doubles(const FwhPlan& pl) { return size_t(pl.ngroups) * pl.Tmax; }

// The kernels of one integration on scratch X / partial (both fully written
// before they are read), then a synchronisation of the stream.
int fwh_run(const FwhPlan& pl, const double* hist, int nt, int npts, const double* y, const double* n,
            const double* dS, const double* obs, int nobs, double Lspan, int ncopies, double* p_out, int cap,
            int* nt_out, double* t0_out, double* X, double* partial, cudaStream_t s) {
    const int64_t nw = int64_t(nt) * npts;
    k_fwh_series<<<unsigned((nw + 255) / 256), 256, 0, s>>>(hist, nt, npts, n, pl.k, X);
    const size_t sm = FWH_SH_BYTES * size_t(pl.group) * ncopies;
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess && sm > 48 * 1024)
        err = cudaFuncSetAttribute(k_fwh_accum, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    for (int o = 0; o < nobs && err == cudaSuccess; ++o) {
        dim3 grid(unsigned(pl.ngroups), unsigned((pl.Tn[o] + 128 * FWH_KO - 1) / (128 * FWH_KO)));
        k_fwh_accum<<<grid, 128, sm, s>>>(X, nt, npts, y, dS, pl.k, obs[o * 3 + 0], obs[o * 3 + 1],
                                          obs[o * 3 + 2], pl.tstart[o], pl.Tn[o], ncopies, Lspan, pl.group,
                                          partial);
        k_fwh_reduce<<<unsigned((pl.Tn[o] + 31) / 32), dim3(32, 32), 0, s>>>(partial, pl.ngroups, pl.Tn[o],
                                                                             p_out + size_t(o) * cap);
        err = cudaGetLastError();
        nt_out[o] = pl.Tn[o];
        t0_out[o] = pl.tstart[o];
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return fr_set_error_from_fwh(FR_ECUDA, cudaGetErrorString(err));
    return FR_OK;
}

}  // namespace

extern "C" int fwh_integrate(const double* hist, int nt, int npts, const double* y, const double* n,
                             const double* dS, double dtau, double tau0, const double* obs, int nobs,
                             const double Minf[3], double c0, double rho0, double p0, double Lspan,
                             int ncopies, double* p_out, int cap, int* nt_out, double* t0_out, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FwhPlan pl;
    int rc = fwh_plan(nt, npts, y, n, dS, hist, dtau, tau0, obs, nobs, Minf, c0, rho0, p0, Lspan, ncopies, p_out,
                      cap, nt_out, t0_out, s, pl);
    if (rc != FR_OK) return rc;
    double *X = nullptr, *partial = nullptr;
    if (cudaMalloc(&X, sizeof(double) * fwh_series_doubles(npts, nt)) != cudaSuccess ||
        cudaMalloc(&partial, sizeof(double) * fwh_partial_doubles(pl)) != cudaSuccess) {
        if (X) cudaFree(X);
        return fr_set_error_from_fwh(FR_ENOMEM, "cannot allocate FW-H scratch");
    }
    rc = fwh_run(pl, hist, nt, npts, y, n, dS, obs, nobs, Lspan, ncopies, p_out, cap, nt_out, t0_out, X, partial, s);
    cudaFree(X);
    cudaFree(partial);
    return rc;
}

// ---------------------------------------------------------------------------
// fwh_integrate_noalloc: the same computation with its scratch (the source
// series and the partial sums) in a fixed file-scope device array, for callers
// that cannot call cudaMalloc/cudaFree.  On the host the array's name is only
// a stand-in, never a device address: every call looks the address up on the
// current device with cudaGetSymbolAddress (which allocates nothing), so the
// address always belongs to the context the kernels run in.

namespace {

constexpr size_t kNoallocScratchDoubles = size_t(1) << 22;  // 32 MiB per device
__device__ __align__(256) double g_fwh_scratch[kNoallocScratchDoubles];

// Device address of g_fwh_scratch in the current device's context.
int noalloc_scratch(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_fwh_scratch);
    if (e != cudaSuccess || !p)
        return fr_set_error_from_fwh(FR_ECUDA, (std::string("cudaGetSymbolAddress of the FW-H scratch: ") +
                                                cudaGetErrorString(e)).c_str());
    *out = static_cast<double*>(p);
    return FR_OK;
}

}  // namespace

extern "C" int fwh_integrate_noalloc(const double* hist, int nt, int npts, const double* y, const double* n,
                                     const double* dS, double dtau, double tau0, const double* obs, int nobs,
                                     const double Minf[3], double c0, double rho0, double p0, double Lspan,
                                     int ncopies, double* p_out, int cap, int* nt_out, double* t0_out,
                                     void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FwhPlan pl;
    int rc = fwh_plan(nt, npts, y, n, dS, hist, dtau, tau0, obs, nobs, Minf, c0, rho0, p0, Lspan, ncopies, p_out,
                      cap, nt_out, t0_out, s, pl);
    if (rc != FR_OK) return rc;
    // the series and the partial rows must fit the fixed scratch
    const size_t need = fwh_series_doubles(npts, nt) + fwh_partial_doubles(pl);
    if (need > kNoallocScratchDoubles)
        return fr_set_error_from_fwh(
            FR_EINVAL, ("fwh_integrate_noalloc: needs " + std::to_string(need) + " doubles of scratch, the fixed "
                        "maximum is " + std::to_string(kNoallocScratchDoubles) +
                        " (8*npts*nt + ceil(npts/max(1,32/ncopies))*window); use fwh_integrate").c_str());
    double* X = nullptr;
    rc = noalloc_scratch(&X);
    if (rc != FR_OK) return rc;
    return fwh_run(pl, hist, nt, npts, y, n, dS, obs, nobs, Lspan, ncopies, p_out, cap, nt_out, t0_out, X,
                   X + fwh_series_doubles(npts, nt), s);
}
