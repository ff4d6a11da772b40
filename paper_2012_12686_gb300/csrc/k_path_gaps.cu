// The fused kernel with per-gap Fresnel propagators (sparse / variable slice spacing, Sec. 2.2)
// and the slice-gap gradient; a translation unit of its own so that it compiles in parallel with
// the uniform-spacing instantiation in k_path.cu.
#include "k_path.cuh"

namespace adorym {

cudaError_t launch_path_gaps(const PathArgs& a, int farfield, cudaStream_t s) {
  switch (a.N) {
#define ADORYM_CASE(n)                                                                    \
  case n:                                                                                 \
    return farfield ? launch_path_t<n, 1, true>(a, s) : launch_path_t<n, 0, true>(a, s);
    ADORYM_CASE(8)
    ADORYM_CASE(16)
    ADORYM_CASE(32)
    ADORYM_CASE(64)
    ADORYM_CASE(128)
#undef ADORYM_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t prepare_path_gaps(int N, int farfield) {
  switch (N) {
    case 8: return farfield ? prepare_path_t<8, 1, true>() : prepare_path_t<8, 0, true>();
    case 16: return farfield ? prepare_path_t<16, 1, true>() : prepare_path_t<16, 0, true>();
    case 32: return farfield ? prepare_path_t<32, 1, true>() : prepare_path_t<32, 0, true>();
    case 64: return farfield ? prepare_path_t<64, 1, true>() : prepare_path_t<64, 0, true>();
    case 128: return farfield ? prepare_path_t<128, 1, true>() : prepare_path_t<128, 0, true>();
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace adorym
