// Cheaper-tail instantiations of the separable-PSF mixed render kernel: the windows with tail
// edges (K >= 3), for models whose widest PSF keeps those edges' arguments within the cheaper
// rational's fit (the plan's far_tails).  A separate translation unit so that the library's
// sets of instantiations compile in parallel.
#include "render_mixed.cuh"

namespace e2e {

cudaError_t launch_render_mixed_far(int K, int DX, int DY, bool check, const MixedArgs& a, const MergeArgs& mg,
                                    int n_items, size_t smem, cudaStream_t st) {
  if (check) return launch_render_mixed_far_checked(K, DX, DY, a, mg, n_items, smem, st);
#define E2E_V(KK, X, Y) \
  if (K == KK && DX == X && DY == Y) return launch_one<KK, X, Y, false, true>(a, mg, n_items, smem, st);
  E2E_MIXED_FAR_VARIANTS(E2E_V)
#undef E2E_V
  return cudaErrorInvalidValue;
}

}  // namespace e2e
