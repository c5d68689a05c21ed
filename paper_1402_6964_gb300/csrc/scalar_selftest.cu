// scalar_selftest.cu -- the Householder scalars of the leaves (hh_scalars)
// evaluated beside the IEEE operations on caller-supplied arguments, so that
// their accuracy can be checked against CUDA's correctly rounded results.
#include "../../include/mrnmf.h"
#include "common.cuh"
#include "internal.h"

namespace mrnmf {
namespace {

__global__ void hh_selftest_kernel(const float* __restrict__ alpha, const float* __restrict__ sig, int64_t count,
                                   float* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float a = alpha[i], s = sig[i];
    const HhScalars h = hh_scalars(a, s);
    const float nrm = sqrtf(fmaf(a, a, s));
    const float beta = a >= 0.f ? -nrm : nrm;
    const float d = a - beta;
    float* o = out + 8 * i;
    o[0] = h.beta;
    o[1] = h.d;
    o[2] = h.rb;
    o[3] = h.rd;
    o[4] = beta;
    o[5] = d;
    o[6] = __frcp_rn(beta);
    o[7] = __frcp_rn(d);
}

}  // namespace
}  // namespace mrnmf

extern "C" mrnmf_status mrnmf_hh_scalars_selftest(const float* alpha, const float* sigma, int64_t count, float* out,
                                                  void* stream)
{
    if (count < 0 || (count > 0 && (!alpha || !sigma || !out))) return MRNMF_ERR_INVALID_ARG;
    if (count == 0) return MRNMF_OK;
    const int threads = 256;
    const int64_t blocks = (count + threads - 1) / threads;
    if (blocks > 0x7fffffff) return MRNMF_ERR_INVALID_ARG;
    mrnmf::hh_selftest_kernel<<<(unsigned)blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(alpha, sigma,
                                                                                                    count, out);
    mrnmf::count_launch();
    return cudaGetLastError() == cudaSuccess ? MRNMF_OK : MRNMF_ERR_CUDA;
}
