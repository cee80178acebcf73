// Host launchers of the reduced-degree element kernels for one (precision,
// dimension) pair; the including translation unit defines FR_REAL and FR_DIM.
#include "fr_reduced.cuh"

namespace frl {

namespace {

template <typename K>
cudaError_t red_prep(K kernel, size_t smem, unsigned long long& done) {
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    // the attribute belongs to the function on the current device: one bit
    // of `done` per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e == cudaSuccess) done |= bit;
    return e;
}

template <int P, int Q>
int red_face_pq(const frk::Red<FR_REAL>& rd, const FR_REAL* u, const FR_REAL* uf, FR_REAL* fvn,
                const frk::Ops<FR_REAL>& op, const frk::Phys<FR_REAL>& ph, const frk::Geo<FR_REAL>& g,
                cudaStream_t s) {
    auto k = frk::k_red_face<FR_DIM, P, Q, FR_REAL>;
    constexpr size_t sm = frk::smem_red<FR_DIM, P, Q, FR_REAL>(true);
    constexpr int W = frk::red_w<FR_DIM, P, Q, FR_REAL>(true);
    static unsigned long long done = 0;
    const cudaError_t e = red_prep(k, sm, done);
    if (e != cudaSuccess) return int(e);
    if (rd.n <= 0) return 0;
    k<<<unsigned((rd.n + W - 1) / W), 32 * W, sm, s>>>(rd, u, uf, fvn, op, ph, g);
    return int(cudaGetLastError());
}

template <int P, int Q, bool V>
int red_resid_pq(const frk::Red<FR_REAL>& rd, const FR_REAL* u, const FR_REAL* uf, const FR_REAL* fvn,
                 const frk::Ops<FR_REAL>& op, const frk::Phys<FR_REAL>& ph, const frk::Geo<FR_REAL>& g,
                 const frk::Stage<FR_REAL>& st, cudaStream_t s) {
    auto k = frk::k_red_resid<FR_DIM, P, Q, FR_REAL, V>;
    constexpr size_t sm = frk::smem_red<FR_DIM, P, Q, FR_REAL>(false);
    constexpr int W = frk::red_w<FR_DIM, P, Q, FR_REAL>(false);
    static unsigned long long done = 0;
    const cudaError_t e = red_prep(k, sm, done);
    if (e != cudaSuccess) return int(e);
    if (rd.n <= 0) return 0;
    k<<<unsigned((rd.n + W - 1) / W), 32 * W, sm, s>>>(rd, u, uf, fvn, op, ph, g, st);
    return int(cudaGetLastError());
}

}  // namespace

// (P, Q) pairs with 0 <= Q < P <= 4
#define FR_RED_DISPATCH(CALL)                                  \
    switch (P * 8 + Q) {                                       \
        case 8: return CALL(1, 0);                             \
        case 16: return CALL(2, 0);                            \
        case 17: return CALL(2, 1);                            \
        case 24: return CALL(3, 0);                            \
        case 25: return CALL(3, 1);                            \
        case 26: return CALL(3, 2);                            \
        case 32: return CALL(4, 0);                            \
        case 33: return CALL(4, 1);                            \
        case 34: return CALL(4, 2);                            \
        case 35: return CALL(4, 3);                            \
        default: return int(cudaErrorInvalidValue);            \
    }

template <>
int red_face<FR_REAL, FR_DIM>(int P, int Q, const frk::Red<FR_REAL>& rd, const FR_REAL* u, const FR_REAL* uf,
                              FR_REAL* fvn, const frk::Ops<FR_REAL>& op, const frk::Phys<FR_REAL>& ph,
                              const frk::Geo<FR_REAL>& g, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
#define C(PP, QQ) red_face_pq<PP, QQ>(rd, u, uf, fvn, op, ph, g, s)
    FR_RED_DISPATCH(C)
#undef C
}

template <>
int red_resid<FR_REAL, FR_DIM>(int P, int Q, const frk::Red<FR_REAL>& rd, const FR_REAL* u, const FR_REAL* uf,
                               const FR_REAL* fvn, const frk::Ops<FR_REAL>& op, const frk::Phys<FR_REAL>& ph,
                               const frk::Geo<FR_REAL>& g, const frk::Stage<FR_REAL>& st, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
#define C(PP, QQ) (ph.viscous ? red_resid_pq<PP, QQ, true>(rd, u, uf, fvn, op, ph, g, st, s) \
                              : red_resid_pq<PP, QQ, false>(rd, u, uf, fvn, op, ph, g, st, s))
    FR_RED_DISPATCH(C)
#undef C
}

#undef FR_RED_DISPATCH

}  // namespace frl
