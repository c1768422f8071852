// Diagnostic entry point: evaluate the renderer's FP32 Gaussian-tail function on given
// arguments, so tests can check it against CUDA's FP64 erfc.
#include "../../include/e2e_render.h"
#include "phi32.cuh"

namespace {

__global__ void k_eval_tail(const double* __restrict__ u, int64_t n, float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = u[i] * e2e::kSqrtLog2eD;  // the kernels' argument is in log2 units
    const float h = (float)v;
    const float l = (float)(v - (double)h);
    out[i] = e2e::tail2(h, l);
  }
}

}  // namespace

extern "C" int e2e_eval_tail(const double* u_dev, int64_t n, float* out_dev, void* stream) {
  if (n < 0 || (n > 0 && (!u_dev || !out_dev))) return E2E_EINVAL;
  if (n == 0) return E2E_OK;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_eval_tail<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(u_dev, n, out_dev);
  return cudaGetLastError() == cudaSuccess ? E2E_OK : E2E_ECUDA;
}
