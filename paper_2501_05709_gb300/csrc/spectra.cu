// Welch power spectral density of observer pressure series (Section 3.3: the
// PSD of the pressure fluctuations by Welch's method with three Hann windows
// and 50% overlap).  Readings, shared with the declaration in fr.h: segment
// length L = 2 floor(nt / (nseg + 1)), step L / 2, periodic Hann window, each
// segment's mean removed, one-sided density averaged over the segments.
//
// Three kernels, all FP64: the table of cos/sin(2 pi m / L); the windowed,
// mean-free segments (one block per observer and segment, fixed-order
// reduction); and a direct DFT with one thread per (observer, frequency) that
// streams each segment through shared memory and walks the twiddle index
// k n mod L incrementally (no modulo, no per-term trigonometry).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "fr.h"

int fr_set_error_from_fwh(int code, const char* msg);

namespace {

__global__ void k_psd_twiddle(int L, double2* __restrict__ cs) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= L) return;
    double s, c;
    sincospi(2.0 * double(m) / double(L), &s, &c);
    cs[m] = make_double2(c, s);
}

// ws[o][s][n] = w_n (x[o][s*step + n] - mean of the segment), w_n = (1 - cos(2 pi n / L)) / 2
__global__ void k_psd_segments(const double* __restrict__ p, int ld, int L, const double2* __restrict__ cs,
                               double* __restrict__ ws) {
    const int s = blockIdx.x, o = blockIdx.y, nseg = gridDim.x;
    const double* x = p + size_t(o) * ld + size_t(s) * (L / 2);
    __shared__ double red[256];
    double acc = 0.0;
    for (int n = threadIdx.x; n < L; n += blockDim.x) acc += x[n];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    const double mean = red[0] / double(L);
    double* out = ws + (size_t(o) * nseg + s) * L;
    for (int n = threadIdx.x; n < L; n += blockDim.x) out[n] = (0.5 - 0.5 * cs[n].x) * (x[n] - mean);
}

constexpr int PSD_TILE = 2048;   // segment samples staged per pass (16 KB)

// psd[o][k] = scale_k * mean over segments of |sum_n ws_n e^{-2 pi i k n / L}|^2
__global__ void k_psd_dft(const double* __restrict__ ws, int nseg, int L, const double2* __restrict__ cs,
                          double inv_norm, double* __restrict__ psd, int cap) {
    __shared__ double tile[PSD_TILE];
    const int o = blockIdx.y;
    const int nf = L / 2 + 1;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    for (int s = 0; s < nseg; ++s) {
        const double* y = ws + (size_t(o) * nseg + s) * L;
        double re = 0.0, im = 0.0;
        int idx = 0;
        for (int n0 = 0; n0 < L; n0 += PSD_TILE) {
            const int cnt = min(PSD_TILE, L - n0);
            __syncthreads();
            for (int n = threadIdx.x; n < cnt; n += blockDim.x) tile[n] = y[n0 + n];
            __syncthreads();
            if (k < nf) {
                for (int n = 0; n < cnt; ++n) {
                    const double2 t = cs[idx];
                    re += tile[n] * t.x;
                    im -= tile[n] * t.y;
                    idx += k;
                    if (idx >= L) idx -= L;
                }
            }
        }
        acc += re * re + im * im;
    }
    if (k < nf) {
        const double c = (k == 0 || 2 * k == L) ? 1.0 : 2.0;
        psd[size_t(o) * cap + k] = c * acc * inv_norm / double(nseg);
    }
}

}  // namespace

extern "C" int fwh_psd(const double* p, int nobs, int nt, int ld, double dt, int nseg, double* psd, int cap,
                       int* nfreq_out, void* stream) {
    if (!p || !psd || !nfreq_out) return fr_set_error_from_fwh(FR_EINVAL, "null argument");
    if (nobs < 1 || nseg < 1 || ld < nt || !(dt > 0.0))
        return fr_set_error_from_fwh(FR_EINVAL, "bad sizes (nobs >= 1, nseg >= 1, ld >= nt, dt > 0 required)");
    const int L = 2 * (nt / (nseg + 1));
    if (L < 2) return fr_set_error_from_fwh(FR_EINVAL, "record too short for the segments");
    const int nf = L / 2 + 1;
    if (cap < nf) return fr_set_error_from_fwh(FR_EINVAL, "output capacity below L/2 + 1 frequencies");
    if (nobs > 65535) return fr_set_error_from_fwh(FR_EINVAL, "too many observers for one launch");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // sum of the squared window, on the host in double
    double w2 = 0.0;
    for (int n = 0; n < L; ++n) {
        const double w = 0.5 - 0.5 * std::cos(2.0 * M_PI * double(n) / double(L));
        w2 += w * w;
    }
    const double inv_norm = dt / w2;   // 1 / (f_s sum w^2)
    double2* cs = nullptr;
    double* ws = nullptr;
    if (cudaMalloc(&cs, sizeof(double2) * size_t(L)) != cudaSuccess ||
        cudaMalloc(&ws, sizeof(double) * size_t(nobs) * nseg * L) != cudaSuccess) {
        cudaFree(cs);
        return fr_set_error_from_fwh(FR_ENOMEM, "cannot allocate PSD scratch");
    }
    k_psd_twiddle<<<(L + 255) / 256, 256, 0, s>>>(L, cs);
    k_psd_segments<<<dim3(nseg, nobs), 256, 0, s>>>(p, ld, L, cs, ws);
    k_psd_dft<<<dim3((nf + 127) / 128, nobs), 128, 0, s>>>(ws, nseg, L, cs, inv_norm, psd, cap);
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    cudaFree(cs);
    cudaFree(ws);
    if (err != cudaSuccess) return fr_set_error_from_fwh(FR_ECUDA, cudaGetErrorString(err));
    *nfreq_out = nf;
    return FR_OK;
}
