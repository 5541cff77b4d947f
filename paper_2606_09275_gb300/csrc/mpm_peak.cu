// Measured FP64 fused multiply-add throughput: the ceiling of the kernels
// that the precision pattern keeps in FP64 (kinematics, the constitutive
// update, the internal-force gather, the basis).  GB300 issues FP64 at a small
// fraction of its FP32 rate, so these kernels are bound by this pipe rather
// than by HBM; their roofline fractions are taken against this measurement.
#include <algorithm>

#include "mpm_internal.cuh"

namespace mpm {
namespace {

constexpr int kChains = 8;

// kChains independent chains x <- x a + b per thread; a < 1 keeps them bounded
__global__ void __launch_bounds__(256) k_fp64_fma(long long iters, double a, double b, double* sink) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1e-3 * (threadIdx.x + 1) + k;
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  if (s == -1.0) sink[blockIdx.x] = s;  // never true; keeps the chains live
}

}  // namespace
}  // namespace mpm

using namespace mpm;

extern "C" int mpm_fp64_peak(mpm_ctx* c, double seconds, double* flops_per_s, double* ms_out) {
  if (!c || !flops_per_s || !(seconds >= 0.05 && seconds <= 10.0)) return MPM_ERR_ARG;
  try {
    cudaStream_t st = c->stream;
    int dev = c->device, nsm = 0;
    MPM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = 0;
    MPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_fma, 256, 0));
    int blocks = nsm * std::max(per_sm, 1);
    double* sink = (double*)c->d_red;
    cudaEvent_t a, b;
    MPM_CUDA(cudaEventCreate(&a));
    MPM_CUDA(cudaEventCreate(&b));
    auto run = [&](long long iters) {
      MPM_CUDA(cudaEventRecord(a, st));
      MPM_LAUNCH(k_fp64_fma<<<blocks, 256, 0, st>>>(iters, 0.9999999, 1e-7, sink));
      MPM_CUDA(cudaEventRecord(b, st));
      MPM_CUDA(cudaEventSynchronize(b));
      float ms = 0.f;
      MPM_CUDA(cudaEventElapsedTime(&ms, a, b));
      return (double)ms;
    };
    run(1000);  // warm-up
    long long iters = 20000;
    double ms = run(iters);
    // scale to the requested duration
    iters = std::max(1000LL, (long long)((double)iters * seconds * 1e3 / std::max(ms, 1e-3)));
    ms = run(iters);
    MPM_CUDA(cudaEventDestroy(a));
    MPM_CUDA(cudaEventDestroy(b));
    double flops = 2.0 * kChains * (double)iters * 256.0 * (double)blocks;
    *flops_per_s = flops / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return MPM_OK;
  } catch (const CudaError& e) {
    set_error(c, e.what());
    return e.code;
  }
}
