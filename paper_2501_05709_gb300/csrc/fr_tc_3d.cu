// Residual kernels of the tensor-core precision modes (FR_TF32_TC,
// FR_BF16X3_TC): float state and point-wise arithmetic as in FR_FP32, with the
// gradient and divergence line operators of k_residual on the tensor cores
// (mma.sync m16n8k8, FP32 accumulation).  3D, orders 3 and 4; the other
// kernels of these modes are the FP32 ones.
#include "fr_kernels.cuh"

namespace frl {

namespace {

template <typename K>
cudaError_t prep_tc(K kernel, size_t smem, unsigned long long& done) {
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

template <int P, int MP, bool VISC, bool BND, int OPM>
int resid_tc_p(const float* u, const float* uf, const float* fvn, int64_t E, const frk::Ops<float>& op,
               const frk::Phys<float>& ph, const frk::Geo<float>& g, const frk::Stage<float>& st, frk::Launch lc,
               cudaStream_t s) {
    auto k = frk::k_residual<3, P, float, MP, VISC, BND, OPM>;
    const size_t sm = frk::smem_resid<3, P, float>(lc.epb, g.sS_sp != 0);
    static unsigned long long done = 0;
    cudaError_t e = prep_tc(k, sm, done);
    if (e != cudaSuccess) return int(e);
    if (E == 0) return 0;
    const unsigned grid = unsigned((E + lc.epb - 1) / lc.epb);
    k<<<grid, frk::Grp<3, P>::T * lc.epb, sm, s>>>(u, uf, fvn, E, op, ph, g, st);
    return int(cudaGetLastError());
}

}  // namespace

int residual_tc3(int P, int opm, const float* u, const float* uf, const float* fvn, int64_t E,
                 const frk::Ops<float>& op, const frk::Phys<float>& ph, const frk::Geo<float>& g,
                 const frk::Stage<float>& st, frk::Launch lc, void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int mp = g.sS_sp != 0 ? 0 : g.diag ? 2 : 1;
#define A(PP, M, V, O) resid_tc_p<PP, M, V, true, O>(u, uf, fvn, E, op, ph, g, st, lc, s)
#define N(PP, M, V, O) resid_tc_p<PP, M, V, false, O>(u, uf, fvn, E, op, ph, g, st, lc, s)
#define R(PP, V, O) (mp == 0 ? A(PP, 0, V, O) : mp == 1 ? (g.bnd ? A(PP, 1, V, O) : N(PP, 1, V, O)) \
                                              : (g.bnd ? A(PP, 2, V, O) : N(PP, 2, V, O)))
#define C(PP, O) (ph.viscous ? R(PP, true, O) : R(PP, false, O))
    if (P == 3) return opm == 1 ? C(3, 1) : C(3, 2);
    if (P == 4) return opm == 1 ? C(4, 1) : C(4, 2);
    return int(cudaErrorInvalidValue);
#undef C
#undef R
#undef N
#undef A
}

}  // namespace frl
