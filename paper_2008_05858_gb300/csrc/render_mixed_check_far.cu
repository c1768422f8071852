// Debug-check instantiations of the cheaper-tail separable render kernel (render_mixed_far.cu):
// the same kernel, also counting every deposit the plan did not foresee.
#include "render_mixed.cuh"

namespace e2e {

cudaError_t launch_render_mixed_far_checked(int K, int DX, int DY, const MixedArgs& a, const MergeArgs& mg,
                                            int n_items, size_t smem, cudaStream_t st) {
#define E2E_V(KK, X, Y) \
  if (K == KK && DX == X && DY == Y) return launch_one<KK, X, Y, true, true>(a, mg, n_items, smem, st);
  E2E_MIXED_FAR_VARIANTS(E2E_V)
#undef E2E_V
  return cudaErrorInvalidValue;
}

}  // namespace e2e
