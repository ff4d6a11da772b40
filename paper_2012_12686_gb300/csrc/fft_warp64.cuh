// 64 x 64 propagation passes that finish each 1-D transform inside one warp.
//
// fft_block.cuh splits a 64-point line into two radix-8 Cooley-Tukey stages (S1/S2 forward,
// S3/S4 on the inverse side) and moves the data between the two stages of a line through the
// shared field, with a CTA barrier after every pass: a propagation step F^-1{F[.] H} costs six
// shared-memory round trips and six barriers, and at N = 64 each pass is short (eight values per
// thread), so the CTA spends most of a step waiting at those barriers.  Here the eight tasks of a
// line (t = 0..7) are eight lanes of one warp.  The slot exchange between the two stages of a
// line goes through a per-warp scratch area with warp-level synchronisation only, and a CTA
// barrier is needed only where the work moves from columns to rows and back:
//   column pass (c14):  y-S3 | exchange | y-S4 | spatial op | y-S1 | exchange | y-S2
//   row pass    (r23):  x-S1 | exchange | x-S2 | frequency op | x-S3 | exchange | x-S4
// Between the passes the field is in shared memory in natural order (row y or y-frequency,
// column x or x-frequency), so a step is two round trips and two barriers; fwd_pair and inv_pair
// have nothing left to do.  Every stage applies the arithmetic of the six-pass scheme (the same
// radix-8 DFT, the same twiddles from the same FP64-built table, in the same order), so both
// schemes give the same values.
//
// Thread roles (512 threads, 16 warps): lane = 4 a + g in warp w works on line 4 w + g (column x
// in the column pass, row in the row pass) as task t = a.  The field's leading dimension is 68
// (4 mod 16 in float2 units): with four consecutive lines per warp and the eight tasks spread
// over the lanes, every 64-bit shared access of a warp in both passes covers all 32 banks (two
// wavefronts), and the global accesses of the spatial ops cover 8 rows x 4 consecutive columns
// (one 32-byte sector per row).
//
// Exchange: after a first stage, lane (a, g) holds in v[k] the slot that task k of the second
// stage takes as its input a.  It stores v[k] at scratch[lane + 36 k] (= g + 4 a + 36 k); lane
// (a', g) then reads v[i] = scratch[g + 4 i + 36 a'].  Both patterns are conflict-free.
#pragma once
#include "fft_block.cuh"
#include "kernels.cuh"

namespace adorym {

struct W64 {
  static constexpr int N = 64, LD = 68, NT = 512;
  static constexpr int SCR_WARP = 288;                    // float2 of exchange scratch per warp
  static constexpr int SCRATCH = (NT / 32) * SCR_WARP;    // float2, placed before the field
  __device__ static __forceinline__ int line() { return 4 * (int)(threadIdx.x >> 5) + (int)(threadIdx.x & 3); }
  __device__ static __forceinline__ int task() { return (int)(threadIdx.x >> 2) & 7; }
};

// slot exchange between the two stages of the lines of one warp (see above)
__device__ __forceinline__ void w64_exchange(float2 (&v)[8], float2* __restrict__ scr) {
  const int lane = (int)(threadIdx.x & 31);
  float2* ws = scr + (threadIdx.x >> 5) * W64::SCR_WARP;
  __syncwarp();   // the previous exchange of this warp has read its slots
#pragma unroll
  for (int k = 0; k < 8; ++k) ws[lane + 36 * k] = v[k];
  __syncwarp();
  const float2* rs = ws + (lane & 3) + 36 * (lane >> 2);
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = rs[4 * i];
}

// One 64-point line transform of sign S: first stage (radix-8 DFT, twiddles W_64^(S t k)),
// exchange, second stage (radix-8 DFT).  Forward (S1, S2): input v[i] = sample 8 i + t, output
// v[i] = frequency t + 8 i.  Inverse side (S3, S4): input v[i] = frequency t + 8 i, output
// v[k] = sample 8 k + t.
// wt[k] = W_64^(t k) (k = 1..7) are the task's twiddles, read once per pass from the shared table:
// the same factors and products as twiddle<S>(v, tw, t).
template <int S>
__device__ __forceinline__ void w64_line(float2 (&v)[8], const float2 (&wt)[8], float2* __restrict__ scr) {
  dft<8, S>(v);
#pragma unroll
  for (int k = 1; k < 8; ++k) v[k] = S < 0 ? cmul(v[k], wt[k]) : cmulc(v[k], wt[k]);
  w64_exchange(v, scr);
  dft<8, S>(v);
}
__device__ __forceinline__ void w64_twiddles(float2 (&wt)[8], const float2* __restrict__ tw, int t) {
#pragma unroll
  for (int k = 1; k < 8; ++k) wt[k] = tw[t * k];
}

// The PathFFT interface (fft_block4.cuh) on the scheme above.  A is the field; the exchange
// scratch lies in the SCRATCH float2 just before it.
struct PathFFTW64 {
  static constexpr int N = 64, LD = W64::LD, SCRATCH = W64::SCRATCH;
  static constexpr int CY = 8, YS = 8, RX = 8, KXS = 8;
  static constexpr bool PAIRS = false;   // fwd_pair and inv_pair are empty
  // column pass: LOAD reads y-frequencies t + 8 i of column x and finishes the inverse y
  // transform (S3, S4) with sign S4; op sees samples y = 8 k + t; STORE runs the forward y
  // transform (S1, S2) with sign S1 and stores y-frequencies t + 8 i
  template <int S4, int S1, bool LOAD, bool STORE, class Pre, class Op>
  __device__ static __forceinline__ void c14(float2* A, const float2* tw, Pre pre, Op op) {
    static_assert(Geo<64>::NT == W64::NT, "the warp-exchange scheme runs 512 threads per CTA");
    static_assert(!LOAD || S4 != 0, "the field between passes is in y-frequency order");
    static_assert(!STORE || S1 != 0, "the field between passes is in y-frequency order");
    const int x = W64::line(), t = W64::task();
    float2* scr = A - SCRATCH;
    float2 pa[8], pb[8], v[8], wt[8];
    pre(pa, pb, x, t);
    w64_twiddles(wt, tw, t);
    if (LOAD) {
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = A[(t + 8 * i) * LD + x];
      w64_line<S4>(v, wt, scr);
    }
    op(v, pa, pb, x, t);
    if (STORE) {
      w64_line<S1>(v, wt, scr);
#pragma unroll
      for (int i = 0; i < 8; ++i) A[(t + 8 * i) * LD + x] = v[i];
    }
  }
  template <int S>
  __device__ static __forceinline__ void fwd_pair(float2*, const float2*) {}
  // row pass on row ky: S2 != 0 reads samples x = 8 i + t and runs the forward x transform; op
  // sees x-frequencies t + 8 i; S3 != 0 runs the inverse x transform and stores samples in place
  template <int S2, int S3, class Op>
  __device__ static __forceinline__ void r23(float2* A, const float2* tw, Op op) {
    const int r = W64::line(), t = W64::task();
    float2* scr = A - SCRATCH;
    float2 v[8], wt[8];
    w64_twiddles(wt, tw, t);
    if (S2) {
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = A[r * LD + 8 * i + t];
      w64_line<S2>(v, wt, scr);
    }
    op(v, r, t);
    if (S3) {
      w64_line<S3>(v, wt, scr);
#pragma unroll
      for (int k = 0; k < 8; ++k) A[r * LD + 8 * k + t] = v[k];
    }
  }
  template <int S>
  __device__ static __forceinline__ void inv_pair(float2*, const float2*) {}
};

}  // namespace adorym
