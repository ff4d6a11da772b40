// The fused kernel with recompute helpers (CTAs beyond the batch recompute checkpoint segments on
// the SMs a batch below the SM count leaves idle); a translation unit of its own so that it
// compiles in parallel with the other instantiations.
#include "k_path.cuh"

namespace adorym {

cudaError_t launch_path_help(const PathArgs& a, int farfield, cudaStream_t s) {
  switch (a.N) {
#define ADORYM_CASE(n)                                                                  \
  case n:                                                                               \
    return farfield ? launch_path_help_t<n, 1>(a, s) : launch_path_help_t<n, 0>(a, s);
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

cudaError_t prepare_path_help(int N, int farfield) {
  switch (N) {
    case 8: return farfield ? prepare_path_help_t<8, 1>() : prepare_path_help_t<8, 0>();
    case 16: return farfield ? prepare_path_help_t<16, 1>() : prepare_path_help_t<16, 0>();
    case 32: return farfield ? prepare_path_help_t<32, 1>() : prepare_path_help_t<32, 0>();
    case 64: return farfield ? prepare_path_help_t<64, 1>() : prepare_path_help_t<64, 0>();
    case 128: return farfield ? prepare_path_help_t<128, 1>() : prepare_path_help_t<128, 0>();
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace adorym
