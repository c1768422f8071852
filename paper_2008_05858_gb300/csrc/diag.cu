// Diagnostic entry points: evaluate the renderer's FP32 Gaussian-tail functions (the general
// one and the cheaper one of narrow PSFs' tail edges) on given arguments, so tests can check
// them against CUDA's FP64 erfc; and a fused multiply-add probe that measures the FP32 and
// FP64 FMA rates the roofline of the ALU-bound kernels is quoted against.
#include "../../include/e2e_render.h"
#include "phi32.cuh"

namespace {

template <bool FAR>
__global__ void k_eval_tail(const double* __restrict__ u, int64_t n, float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = u[i] * e2e::kSqrtLog2eD;  // the kernels' argument is in log2 units
    const float h = (float)v;
    const float l = (float)(v - (double)h);
    out[i] = FAR ? e2e::tail2_far(h, l) : e2e::tail2(h, l);
  }
}

int eval_tail(bool far, const double* u_dev, int64_t n, float* out_dev, void* stream) {
  if (n < 0 || (n > 0 && (!u_dev || !out_dev))) return E2E_EINVAL;
  if (n == 0) return E2E_OK;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (far)
    k_eval_tail<true><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(u_dev, n, out_dev);
  else
    k_eval_tail<false><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(u_dev, n, out_dev);
  return cudaGetLastError() == cudaSuccess ? E2E_OK : E2E_ECUDA;
}

// Each thread runs kChains independent FMA chains of `iters` steps (no chain waits on another,
// so the pipe, not latency, sets the rate) and stores their sum, which keeps them live.
constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T a, T b, T* __restrict__ sink) {
  T v[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) v[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = v[c] * a + b;  // contracted to one FMA
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += v[c];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int e2e_fma_probe(int32_t fp64, int32_t blocks, int32_t iters, void* sink_dev, int64_t* fmas,
                             void* stream) {
  if (blocks < 1 || iters < 1 || !sink_dev || !fmas) return E2E_EINVAL;
  const cudaStream_t st = (cudaStream_t)stream;
  if (fp64)
    k_fma_probe<double><<<blocks, 256, 0, st>>>(iters, 0.999999, 1e-7, static_cast<double*>(sink_dev));
  else
    k_fma_probe<float><<<blocks, 256, 0, st>>>(iters, 0.999999f, 1e-7f, static_cast<float*>(sink_dev));
  *fmas = (int64_t)blocks * 256 * iters * kChains;
  return cudaGetLastError() == cudaSuccess ? E2E_OK : E2E_ECUDA;
}

extern "C" int e2e_eval_tail(const double* u_dev, int64_t n, float* out_dev, void* stream) {
  return eval_tail(false, u_dev, n, out_dev, stream);
}

extern "C" int e2e_eval_tail_far(const double* u_dev, int64_t n, float* out_dev, void* stream) {
  return eval_tail(true, u_dev, n, out_dev, stream);
}
