// Host launchers of the FR kernels for one (precision, dimension) pair; the
// including translation unit defines FR_REAL and FR_DIM.
#include "fr_kernels.cuh"

#include <algorithm>

namespace frl {

namespace {

// Opt every kernel in to the full 227 KB of dynamic shared memory on its first
// use (a launch with E == 0 does only this), so that later launches of any
// tile size, including those recorded into a CUDA graph, need no attribute call.
// `done` belongs to the caller's own kernel instantiation (kernels of
// different orders share a signature, so the flag cannot live here).
template <typename K>
cudaError_t prep(K kernel, size_t smem, unsigned long long& done) {
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    // the attribute belongs to the function on the current device: one bit
    // of `done` per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    // and to the largest shared-memory carveout: left to itself the driver
    // configured too little shared memory for the blocks that the registers
    // admit (four blocks per SM at p = 4 in 3D where five or six fit)
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 int(cudaSharedmemCarveoutMaxShared));
    if (e == cudaSuccess) done |= bit;
    return e;
}

inline unsigned grid_of(int64_t E, int epb) { return unsigned((E + epb - 1) / epb); }

template <int P>
int traces_p(const FR_REAL* u, FR_REAL* uf, int64_t E, const frk::Ops<FR_REAL>& op, frk::Launch lc,
             cudaStream_t s) {
    auto k = frk::k_traces<FR_DIM, P, FR_REAL>;
    const size_t sm = frk::smem_traces<FR_DIM, P, FR_REAL>(lc.epb);
    static unsigned long long done = 0;
    cudaError_t e = prep(k, sm, done);
    if (e != cudaSuccess) return int(e);
    if (E == 0) return 0;
    k<<<grid_of(E, lc.epb), frk::Grp<FR_DIM, P>::T * lc.epb, sm, s>>>(u, uf, E, op);
    return int(cudaGetLastError());
}

// metric path of the kernels: 0 per-point metrics, 1 affine, 2 affine with diagonal S
inline int metric_path(const frk::Geo<FR_REAL>& g) { return g.sS_sp != 0 ? 0 : g.diag ? 2 : 1; }

// Blocks of a persistent launch: as many as fit on every SM at once (threads,
// registers in units of 8 per thread, shared memory with 1 KB reserved per
// block), at most one per tile of elements.
inline unsigned persistent_grid(int64_t E, int epb, int threads, size_t smem, int regs, int nsm) {
    const int r8 = (std::max(regs, 1) + 7) / 8 * 8;
    int per = std::min(2048 / threads, 32);
    per = std::min(per, 65536 / (threads * r8));
    per = std::min(per, int(233472 / (smem + 1024)));
    const int64_t cap = int64_t(std::max(per, 1)) * std::max(nsm, 1);
    return unsigned(std::min<int64_t>(int64_t(grid_of(E, epb)), cap));
}

template <int P, int MP, bool BND>
int visc_p(const FR_REAL* u, const FR_REAL* uf, FR_REAL* fvn, int64_t E, const frk::Ops<FR_REAL>& op,
           const frk::Phys<FR_REAL>& ph, const frk::Geo<FR_REAL>& g, frk::Launch lc, cudaStream_t s) {
    if constexpr (MP == 0) {
        auto k = frk::k_visc_face<FR_DIM, P, FR_REAL, MP, BND>;
        const size_t sm = frk::smem_visc<FR_DIM, P, FR_REAL>(lc.epb, true);
        static unsigned long long done = 0;
        cudaError_t e = prep(k, sm, done);
        if (e != cudaSuccess) return int(e);
        if (E == 0) return 0;
        k<<<grid_of(E, lc.epb), frk::Grp<FR_DIM, P>::T * lc.epb, sm, s>>>(u, uf, fvn, E, op, ph, g);
        return int(cudaGetLastError());
    } else {
        // affine meshes: the pipelined kernel on a persistent grid, sized from
        // the kernel's registers and the SM count read at set-up (the first,
        // empty launch at mesh load, outside any stream capture)
        auto k = frk::k_visc_face_aff<FR_DIM, P, FR_REAL, MP, BND>;
        const size_t sm = frk::smem_visc<FR_DIM, P, FR_REAL>(lc.epb, false);
        static unsigned long long done = 0;
        static int regs = 0, nsm = 0;
        cudaError_t e = prep(k, sm, done);
        if (e != cudaSuccess) return int(e);
        if (!regs) {
            cudaFuncAttributes fa;
            int dev = 0;
            if ((e = cudaFuncGetAttributes(&fa, k)) != cudaSuccess) return int(e);
            if ((e = cudaGetDevice(&dev)) != cudaSuccess) return int(e);
            if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return int(e);
            regs = fa.numRegs;
        }
        if (E == 0) return 0;
        const int threads = frk::Grp<FR_DIM, P>::T * lc.epb;
        k<<<persistent_grid(E, lc.epb, threads, sm, regs, nsm), threads, sm, s>>>(u, uf, fvn, E, op, ph, g);
        return int(cudaGetLastError());
    }
}

template <int P, int MP, bool VISC, bool BND>
int resid_p(const FR_REAL* u, const FR_REAL* uf, const FR_REAL* fvn, int64_t E,
            const frk::Ops<FR_REAL>& op, const frk::Phys<FR_REAL>& ph, const frk::Geo<FR_REAL>& g,
            const frk::Stage<FR_REAL>& st, frk::Launch lc, cudaStream_t s) {
    auto k = frk::k_residual<FR_DIM, P, FR_REAL, MP, VISC, BND>;
    const size_t sm = frk::smem_resid<FR_DIM, P, FR_REAL>(lc.epb, g.sS_sp != 0);
    static unsigned long long done = 0;
    cudaError_t e = prep(k, sm, done);
    if (e != cudaSuccess) return int(e);
    if (E == 0) return 0;
    k<<<grid_of(E, lc.epb), frk::Grp<FR_DIM, P>::T * lc.epb, sm, s>>>(u, uf, fvn, E, op, ph, g, st);
    return int(cudaGetLastError());
}

}  // namespace

#define FR_DISPATCH(CALL)                 \
    switch (P) {                          \
        case 1: return CALL(1);           \
        case 2: return CALL(2);           \
        case 3: return CALL(3);           \
        case 4: return CALL(4);           \
        default: return int(cudaErrorInvalidValue); \
    }

template <>
int traces<FR_REAL, FR_DIM>(int P, const FR_REAL* u, FR_REAL* uf, int64_t E, const frk::Ops<FR_REAL>& op,
                            frk::Launch lc, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
#define C(PP) traces_p<PP>(u, uf, E, op, lc, s)
    FR_DISPATCH(C)
#undef C
}

template <>
int visc_face<FR_REAL, FR_DIM>(int P, const FR_REAL* u, const FR_REAL* uf, FR_REAL* fvn, int64_t E,
                               const frk::Ops<FR_REAL>& op, const frk::Phys<FR_REAL>& ph,
                               const frk::Geo<FR_REAL>& g, frk::Launch lc, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int mp = metric_path(g);
    // curved meshes always take the boundary-aware kernels
#define V(PP, M) (g.bnd ? visc_p<PP, M, true>(u, uf, fvn, E, op, ph, g, lc, s) \
                        : visc_p<PP, M, false>(u, uf, fvn, E, op, ph, g, lc, s))
#define C(PP) (mp == 0 ? visc_p<PP, 0, true>(u, uf, fvn, E, op, ph, g, lc, s) : mp == 1 ? V(PP, 1) : V(PP, 2))
    FR_DISPATCH(C)
#undef C
#undef V
}

template <>
int residual<FR_REAL, FR_DIM>(int P, const FR_REAL* u, const FR_REAL* uf, const FR_REAL* fvn, int64_t E,
                              const frk::Ops<FR_REAL>& op, const frk::Phys<FR_REAL>& ph,
                              const frk::Geo<FR_REAL>& g, const frk::Stage<FR_REAL>& st, frk::Launch lc,
                              void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int mp = metric_path(g);
#define B(PP, M, V) (g.bnd ? resid_p<PP, M, V, true>(u, uf, fvn, E, op, ph, g, st, lc, s) \
                           : resid_p<PP, M, V, false>(u, uf, fvn, E, op, ph, g, st, lc, s))
#define R(PP, V) (mp == 0 ? resid_p<PP, 0, V, true>(u, uf, fvn, E, op, ph, g, st, lc, s) \
                  : mp == 1 ? B(PP, 1, V) : B(PP, 2, V))
#define C(PP) (ph.viscous ? R(PP, true) : R(PP, false))
    FR_DISPATCH(C)
#undef C
#undef R
#undef B
}

template <>
int threads_per_element<FR_REAL, FR_DIM>(int P) {
    switch (P) {
        case 1: return frk::Grp<FR_DIM, 1>::T;
        case 2: return frk::Grp<FR_DIM, 2>::T;
        case 3: return frk::Grp<FR_DIM, 3>::T;
        case 4: return frk::Grp<FR_DIM, 4>::T;
        default: return 32;
    }
}

template <>
size_t smem_bytes<FR_REAL, FR_DIM>(int P, int kernel, int epb, bool curved) {
#define C(PP) (kernel == 0 ? frk::smem_traces<FR_DIM, PP, FR_REAL>(epb)          \
               : kernel == 1 ? frk::smem_visc<FR_DIM, PP, FR_REAL>(epb, curved)  \
                             : frk::smem_resid<FR_DIM, PP, FR_REAL>(epb, curved))
    switch (P) {
        case 1: return C(1);
        case 2: return C(2);
        case 3: return C(3);
        case 4: return C(4);
        default: return 0;
    }
#undef C
}

template <>
int forces<FR_REAL, FR_DIM>(int P, const FR_REAL* uf, const FR_REAL* fvn, const int32_t* wall_ef,
                            const int64_t* wall_off, int ncand, const frk::Ops<FR_REAL>& op,
                            const frk::Geo<FR_REAL>& g, FR_REAL gm1, int viscous, double* part, double* fnow,
                            double* fsum, double* fcnt, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (ncand <= 0) return 0;
    const dim3 grid(frk::FORCE_BLOCKS, unsigned(ncand));
#define C(PP) (frk::k_forces<FR_DIM, PP, FR_REAL><<<grid, 256, 0, s>>>(uf, fvn, wall_ef, wall_off, op, g, gm1, \
                                                                        viscous, part),                      \
               frk::k_forces_fin<<<ncand, 32, 0, s>>>(part, frk::FORCE_BLOCKS, fnow, fsum, fcnt),          \
               int(cudaGetLastError()))
    FR_DISPATCH(C)
#undef C
}

template <>
int sample<FR_REAL, FR_DIM>(int P, const FR_REAL* u, const int64_t* pe, const FR_REAL* pw, int npts,
                            const frk::Phys<FR_REAL>& ph, FR_REAL* hist, int* count, int cap, int every,
                            void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const unsigned blocks = unsigned((int64_t(npts) * 32 + 255) / 256);
#define C(PP) ((npts > 0 ? (frk::k_sample<FR_DIM, PP, FR_REAL><<<blocks, 256, 0, s>>>(u, pe, pw, npts, ph, hist, \
                                                                                  count, cap, every), 0) : 0), \
               frk::k_bump<<<1, 32, 0, s>>>(count, cap, every), int(cudaGetLastError()))
    FR_DISPATCH(C)
#undef C
}

template <>
int integrals<FR_REAL, FR_DIM>(int P, const FR_REAL* u, int64_t e_first, int64_t ne,
                               const frk::Ops<FR_REAL>& op, const frk::Geo<FR_REAL>& g, double* partial,
                               int nblocks, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
#define C(PP) (frk::k_integrals<FR_DIM, PP, FR_REAL><<<nblocks, 256, 0, s>>>(u, e_first, ne, op, g, partial), \
               int(cudaGetLastError()))
    FR_DISPATCH(C)
#undef C
}

template <>
int source_stage<FR_REAL, FR_DIM>(int P, const frk::Src<FR_REAL>& src, const frk::Stage<FR_REAL>& st,
                                  const frk::Ops<FR_REAL>& op, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (src.nentry <= 0) return 0;
    const unsigned blocks = unsigned((src.nentry + 3) / 4);
#define C(PP) (frk::k_source_stage<FR_DIM, PP, FR_REAL><<<blocks, 128,                                    \
                   4 * frk::Sz<FR_DIM, PP>::NV * frk::Sz<FR_DIM, PP>::NSP * sizeof(FR_REAL), s>>>(src, st, op),                   \
               int(cudaGetLastError()))
    FR_DISPATCH(C)
#undef C
}

template <>
int sponge<FR_REAL, FR_DIM>(int P, const frk::Sponge<FR_REAL>& sp, FR_REAL* a, FR_REAL* b, FR_REAL* uf_out,
                            const frk::Ops<FR_REAL>& op, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (sp.n <= 0) return 0;
    const unsigned blocks = unsigned((sp.n + 3) / 4);
#define C(PP) (frk::k_sponge<FR_DIM, PP, FR_REAL><<<blocks, 128,                                             \
                   8 * frk::Sz<FR_DIM, PP>::NV * frk::Sz<FR_DIM, PP>::NSP * sizeof(FR_REAL), s>>>(sp, a, b, \
                                                                                              uf_out, op), \
               int(cudaGetLastError()))
    FR_DISPATCH(C)
#undef C
}

template <>
int cfl<FR_REAL, FR_DIM>(int P, const FR_REAL* u, const FR_REAL* hlen, int64_t E, const int64_t* cand_off,
                         int ncand, const frk::Phys<FR_REAL>& ph, unsigned long long* lam, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (E == 0) return 0;
    const unsigned blocks = unsigned((E + 7) / 8);
#define C(PP) (frk::k_cfl<FR_DIM, PP, FR_REAL><<<blocks, 256, 0, s>>>(u, hlen, E, cand_off, ncand, ph, lam), \
               int(cudaGetLastError()))
    FR_DISPATCH(C)
#undef C
}

#undef FR_DISPATCH

}  // namespace frl
