// Arithmetic-peak probe (fk_fma_probe): a grid of independent multiply-add
// chains in FP32 or FP64 on the CUDA cores, for measuring the rate the
// CUDA-core kernels of this library are compared against.  Every thread runs
// CHAINS independent chains a <- a * b + c for `iters` steps; the values
// never reach the (impossible) sink condition, but the compiler cannot know
// that, so no chain is removed.
#include "fk_internal.h"

namespace fk {
namespace {

constexpr int CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T *__restrict__ sink) {
    T a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    const T b = (T)0.999999, c = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    if (s == (T)-12345.0) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace fk

extern "C" int fk_fma_probe(int prec, int blocks, int iters, void *sink, fk_stream stream) {
    using namespace fk;
    if ((prec != FK_FP32 && prec != FK_FP64) || blocks < 1 || iters < 1 || !sink)
        return fail(FK_EINVAL, "fk_fma_probe: prec must be FK_FP32 or FK_FP64, blocks and iters >= 1, sink not NULL");
    const cudaStream_t s = (cudaStream_t)stream;
    if (prec == FK_FP64)
        k_fma_probe<double><<<blocks, 256, 0, s>>>(iters, (double *)sink);
    else
        k_fma_probe<float><<<blocks, 256, 0, s>>>(iters, (float *)sink);
    count_launch();
    FK_CUDA(cudaGetLastError());
    return FK_OK;
}
